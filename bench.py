"""Benchmark: ICCG time to 1e-8 relative residual on the 3D 7-point Poisson
problem (128^3, n = 2,097,152, 14.58M nonzeros, b ~ U[-1,1] from seed 0) with
Leiden CPM blocking (resolution 0.5) and greedy block coloring: the fastest
blocking on a GB300 of the swept set (ABMC block sizes 8..128, Leiden
modularity, CPM resolutions 0.01..0.5).  The default computes the Leiden
blocking on the device with the library's parallel Leiden (the reference arm
computes the same partition with the oracle's sequential statement of it);
`--blocking leiden_cpm` takes the sequential Leiden of the host instead, and
`--blocking abmc --block-size S` an ABMC blocking.
`--workload diffusion96 --fp32` runs the 27-point variable-coefficient
diffusion problem (96^3, ABMC 32) with the FP32 preconditioner (extension 1).
`--workload batch64` runs the batched extension: 64 shifted 7-point systems
(sides U{16..64}), 16 right-hand sides each, ABMC 32, FP32 preconditioner,
all in one launch; a step is the whole batch solved to 1e-8.
`--workload learned` selects and trains the learned-blocking MLP ensemble on
the GPU (library kernels) from the committed label sweep and solves every
held-out matrix live with the predicted ABMC block size and the predicted CPM
resolution, the best constant settings and the fixed settings; a step is the
held-out set solved once with the predicted ABMC block size.

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
workload: each step is the oracle's full solve, IC(0) plus PCG to the
tolerance (about 9 s at 128^3).

The default line also carries extension 1 (the FP32-preconditioner solve of
the same system: time, iterations, error against the FP64 solve and the
oracle) and a compact extension 2 figure (8 systems of config 4's recipe x 16
right-hand sides in one launch, against the plain FP64 solver); --no-ext
leaves them out.
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
               "Laplacians, 3-dof spring networks; n 1e5-2e6), ABMC block size and CPM resolution predicted by the "
               "learned-blocking MLP ensemble",
}


def workload(args):
    if args.workload == "diffusion96":
        a, b, _ = gen.config3(nx=args.nx, seed=args.seed)
        return a, b
    a, b, _ = gen.config2(nx=args.nx, seed=args.seed)
    return a, b


def workload_string(args, a, bl):
    """The workload as both arms name it (same text: same configuration)."""
    seed_b = args.seed + 1 if args.workload == "diffusion96" else args.seed
    return (WORKLOADS[args.workload].format(nx=args.nx) + f" (n={a.n}, nnz={a.nnz}), b~U[-1,1] seed {seed_b}, "
            f"{blocking_name(args)}{'' if args.blocking == 'levels' and not args.split_levels else ' + greedy coloring'} "
            f"(n_b={bl['n_b']}, n_c={bl['n_c']}), "
            f"IC(0) + PCG to {args.tol:g}" + (", FP32 preconditioner" if args.fp32 else ""))


def code_only(src):
    """C++ source without its comments, trailing blanks and empty lines (string
    literals kept), so that a change of comments alone keeps the digest."""
    import re
    tok = re.compile(r'//[^\n]*|/\*.*?\*/|"(?:\\.|[^"\\\n])*"|\'(?:\\.|[^\'\\\n])*\'', re.S)
    out = tok.sub(lambda m: "" if m.group(0)[0] == "/" else m.group(0), src)
    return "\n".join(ln.rstrip() for ln in out.split("\n") if ln.strip())


def kernels_sha():
    """sha256 of the CUDA sources the substitution kernels are built from
    (their code, comments left out)."""
    import hashlib
    h = hashlib.sha256()
    for f in ("kernels.cu", "iccg_internal.h"):
        src = open(os.path.join(ROOT, "paper_2609_00561_gb300", "csrc", f), encoding="utf-8").read()
        h.update(code_only(src).encode())
    return h.hexdigest()


def measured_traffic(key):
    """DRAM bytes (read + write) per PCG iteration of the substitution sweep
    from the committed ncu summary (profiles/subst_traffic.json), or None when
    there is none for this workload or the kernels changed since the capture."""
    path = os.path.join(ROOT, "profiles", "subst_traffic.json")
    if not os.path.exists(path):
        return None, "no capture"
    d = json.load(open(path))
    if d.get("kernels_sha256") != kernels_sha():
        return None, "kernels changed since the last capture"
    e = d.get("entries", {}).get(key)
    if e is None:
        return None, "no capture of this workload"
    return int(e["subst_bytes_per_iteration"]), e.get("how", "ncu")


def make_blocking(mod, a, args):
    """The configured blocking by `mod` (the library, or the oracle for the
    reference arm; both give the same permutation), with blocks above
    --split-levels rows split into in-block levels when asked."""
    if args.blocking == "abmc":
        bl = mod.blocking(a, "abmc", args.block_size)
    elif args.blocking == "levels":
        bl = mod.blocking(a, "levels")
    elif args.blocking.endswith("_par"):
        # the parallel Leiden: on the device in the GPU arm, its sequential
        # statement in the oracle for the reference arm (the same partition)
        method = args.blocking[:-4]
        if hasattr(mod, "dev_blocking"):
            bl = mod.dev_blocking(a, method, args.gamma)
        else:
            q = "cpm" if method == "leiden_cpm" else "modularity"
            gptr, gadj = mod.graph(a.n, a.rowptr, a.colind)
            raw, nb = mod.par_leiden(a.n, gptr, gadj, q, args.gamma)
            block_of = mod.sort_blocks_desc(a.n, nb, raw)
            color_of, nc = mod.color_blocks(a.n, gptr, gadj, nb, block_of)
            perm, bptr, cptr = mod.order(a.n, nb, nc, block_of, color_of)
            bl = {"perm": perm, "block_ptr": bptr, "color_ptr": cptr, "n_b": nb, "n_c": nc,
                  "block_of": block_of, "color_of": color_of}
    else:
        bl = mod.blocking(a, args.blocking, gamma=args.gamma)
    if args.split_levels:
        bl = mod.iccg_split_levels(a, bl, args.split_levels) if hasattr(mod, "iccg_split_levels") \
            else mod.split_levels(a, bl, args.split_levels)
    return bl


def blocking_name(args):
    if args.split_levels:
        return _blocking_name(args) + f", blocks above {args.split_levels} rows split into in-block levels"
    return _blocking_name(args)


def _blocking_name(args):
    if args.blocking == "abmc":
        return f"ABMC s={args.block_size}"
    if args.blocking == "levels":
        return "level sets of the natural order (level scheduling, a color per level)"
    if args.blocking == "leiden_cpm":
        return f"Leiden CPM resolution {args.gamma:g}"
    if args.blocking == "leiden_cpm_par":
        return f"parallel Leiden CPM resolution {args.gamma:g}"
    if args.blocking == "leiden_md_par":
        return f"parallel Leiden modularity resolution {args.gamma:g}"
    return f"Leiden modularity resolution {args.gamma:g}"


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


def hbm_peak():
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peaks = json.load(open(pk_path)) if os.path.exists(pk_path) else {}
    return float(peaks.get("hbm_gbs", 6800.0)), ("measured" if "hbm_gbs" in peaks else "fallback")


def time_steps(step, steps, stream, per_step=None):
    """Device time per step (CUDA events on the launching stream; an event
    after every step, so `per_step`, when a list, receives each step's ms)."""
    import torch
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    torch.cuda.synchronize()
    evs[0].record(stream)
    out = None
    for k in range(steps):
        out = step()
        evs[k + 1].record(stream)
    torch.cuda.synchronize()
    if per_step is not None:
        per_step.extend(evs[k].elapsed_time(evs[k + 1]) for k in range(steps))
    return evs[0].elapsed_time(evs[steps]) / steps, out


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
                    stream=stream.cuda_stream, factor=False, no_graph=args.no_graph, lane_block_max=args.lane_max,
                    tile_mapping=args.tile_mapping, fuse_sweep=args.fuse_sweep)
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
    step_ms = []
    with ClockSampler(local) as clk:
        ms, (st, iters, _) = time_steps(step, args.steps, stream, step_ms)
    if world > 1:
        ms = max_over_ranks(ms, dev)

    # solve alone and factor alone (same inputs, device events)
    factor_ms, _ = time_steps(lambda: iccg.iccg_factor(S.ctx), max(1, args.steps), stream)
    solve_reps = max(1, min(args.steps, 5))

    def solve_once():
        xd.zero_()
        return iccg.iccg_solve(S.ctx, bd, xd, args.tol, args.maxit, want_hist=False)

    solve_ms, (st, iters, _) = time_steps(solve_once, solve_reps, stream)
    x = xd.cpu().numpy()
    true_rel = float(np.linalg.norm(b - a.to_scipy() @ x) / np.linalg.norm(b))

    # roofline of the substitution sweep from the graph-timed solve: an
    # iteration's time minus its SpMV phase (p update + SpMV, event-timed in
    # the same launch configuration); the solve start (one extra sweep, the
    # residual SpMV, permutations) is charged to the sweep as well
    spmv_phase_ms = iccg.iccg_time_spmv_phase(S.ctx, 50)
    sweep_ms_it = solve_ms / max(iters, 1) - spmv_phase_ms
    bm = bytes_model(info["n"], info["nnz"], info["nL"], args.fp32)
    peak, peak_src = hbm_peak()
    achieved = bm["subst"] / (sweep_ms_it * 1e-3) / 1e9 if sweep_ms_it > 0 else 0.0
    it_achieved = bm["total"] * iters / (solve_ms * 1e-3) / 1e9
    tkey = f"{args.workload}|{args.nx}|{blocking_name(args)}|{'fp32' if args.fp32 else 'fp64'}"
    traffic, traffic_src = measured_traffic(tkey)

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

    # the library's own count of the kernels one iccg_factor and one
    # iccg_solve of `iters` iterations launch
    launches_per_step = info["factor_launches"] + info["solve_fixed_launches"] + iters * info["launches_per_iteration"]
    result = {
        "metric": "ICCG time to 1e-8 rel. residual",
        "value": round(ms, 4),
        "unit": "ms",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms, 4),
        "ms_std": round(statistics.pstdev(step_ms), 4) if len(step_ms) > 1 else 0.0,
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64" if args.fp32 else "f64",
        "data": "synthetic",
        "config": {"workload": workload_string(args, a, bl),
                   "step": "iccg_factor + iccg_solve, inputs resident",
                   "l2": "inputs larger than L2 (matrix + factors > 129 MB)",
                   "parallelism": "replicas only" if world > 1 else "1 GPU",
                   "layout": f"{info['tile_colors']} of {info['n_c']} colors as lane tiles ({info['tiles']} tiles), "
                             f"{info['unit_colors']} as warp units, {info['groups']} CTA groups"},
        "iterations": iters,
        "status": iccg.STATUS.get(st, st),
        "true_relres": true_rel,
        "solve_ms": round(solve_ms, 4),
        "factor_ms": round(factor_ms, 4),
        "us_per_iteration": round(solve_ms * 1e3 / max(iters, 1), 2),
        "setup": {"gen_s": round(t_gen, 3), "blocking_s": round(t_block, 3), "setup_s": round(t_setup, 3)},
        "per_iteration_us": {"spmv_phase": round(spmv_phase_ms * 1e3, 2), "sweep": round(sweep_ms_it * 1e3, 2),
                             "how": "sweep = graph-timed solve / iterations - event-timed SpMV phase"},
        "roofline": {"bound": "hbm", "kernel": "block-multicolor substitution sweep (forward, fused and backward "
                                               "color launches of one PCG iteration)",
                     "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "peak_source": peak_src,
                     "bytes_per_iteration": bm["subst"], "traffic": traffic, "traffic_source": traffic_src,
                     "traffic_unit": "DRAM bytes per PCG iteration (ncu, cold cache)"},
        "iteration_roofline": {"bytes_per_iteration": bm["total"], "achieved": round(it_achieved, 1),
                               "frac": round(it_achieved / peak, 4)},
        "e2e": {"value": round(e2e_ms, 4), "unit": "ms", "h2d_bytes_per_step": 2 * 8 * a.n,
                "d2h_bytes_per_step": 8 * a.n},
        "gpu_launches": int(launches_per_step * args.steps),
        "clocks": clk.summary(),
    }
    if not args.no_ext and not args.fp32 and args.workload in ("poisson128", "diffusion96"):
        result["ext_fp32_preconditioner"] = ext_fp32(args, a, b, bl, x, ms, stream, dev)
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        cb, xo, it_o = cpu_baseline(a, b, bl, args)
        result["cpu_baseline"] = cb
        result["parity_vs_oracle"] = {"oracle_iterations": it_o, "iterations": iters,
                                      "rel_error": float(np.linalg.norm(x - xo) / np.linalg.norm(xo)),
                                      "bar": "rel. error <= 1e-10, iterations +-1"}
        if "ext_fp32_preconditioner" in result:
            xf = result["ext_fp32_preconditioner"].pop("_x")
            result["ext_fp32_preconditioner"]["rel_error_vs_oracle"] = float(
                np.linalg.norm(xf - xo) / np.linalg.norm(xo))
    if "ext_fp32_preconditioner" in result:
        result["ext_fp32_preconditioner"].pop("_x", None)
    S.close()
    if not args.no_ext and world == 1 and args.blocking in ("leiden_cpm", "leiden_md") and not args.split_levels:
        result["ext_device_blocking"] = ext_device_blocking(args, a, b, ms, iters, stream, dev)
    if not args.no_ext and world == 1 and args.blocking in ("leiden_cpm_par", "leiden_md_par"):
        result["ext_sequential_leiden"] = ext_sequential_leiden(args, a, b, ms, iters, t_block, stream, dev)
    if not args.no_ext and world == 1 and args.workload == "poisson128":
        result["ext_batched"] = ext_batched(args, stream, dev)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(result))


def ext_device_blocking(args, a, b, ms_host, it_host, stream, dev):
    """The same Leiden blocking computed on the device (graph, parallel
    Leiden, size order, greedy coloring, ordering), its time against the
    host's, and the step (IC(0) + solve) with that blocking."""
    import torch
    from paper_2609_00561_gb300 import iccg
    iccg.dev_blocking(a, args.blocking, args.gamma, stream=stream.cuda_stream)   # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    bl = iccg.dev_blocking(a, args.blocking, args.gamma, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    t_dev = time.perf_counter() - t0
    S = iccg.Solver(a, bl, stream=stream.cuda_stream, factor=False)
    bd = torch.tensor(b, device=dev)
    xd = torch.zeros_like(bd)

    def step():
        iccg.iccg_factor(S.ctx)
        xd.zero_()
        return iccg.iccg_solve(S.ctx, bd, xd, args.tol, args.maxit, want_hist=False)

    for _ in range(max(1, args.warmup)):
        step()
    ms, (st, it, _) = time_steps(step, args.steps, stream)
    x = xd.cpu().numpy()
    S.close()
    return {"blocking_s": round(t_dev, 4), "n_b": int(bl["n_b"]), "n_c": int(bl["n_c"]),
            "ms_per_step": round(ms, 4), "iterations": it, "status": iccg.STATUS.get(st, st),
            "true_relres": float(np.linalg.norm(b - a.to_scipy() @ x) / np.linalg.norm(b)),
            "vs_host_blocking": {"ms_per_step": round(ms_host, 4), "iterations": it_host},
            "how": "wall time of the device pipeline (synchronised), second call"}


def ext_sequential_leiden(args, a, b, ms_par, it_par, t_par, stream, dev):
    """The same resolution with the sequential Leiden on the host (the
    published algorithm's order: random visiting queue, randomized
    refinement): its blocking time and the step with its blocking, next to
    the parallel Leiden's."""
    import torch
    from paper_2609_00561_gb300 import iccg
    method = args.blocking[:-4]
    t0 = time.perf_counter()
    bl = iccg.blocking(a, method, gamma=args.gamma)
    t_host = time.perf_counter() - t0
    S = iccg.Solver(a, bl, stream=stream.cuda_stream, factor=False)
    bd = torch.tensor(b, device=dev)
    xd = torch.zeros_like(bd)

    def step():
        iccg.iccg_factor(S.ctx)
        xd.zero_()
        return iccg.iccg_solve(S.ctx, bd, xd, args.tol, args.maxit, want_hist=False)

    for _ in range(max(1, args.warmup)):
        step()
    ms, (st, it, _) = time_steps(step, args.steps, stream)
    x = xd.cpu().numpy()
    S.close()
    return {"blocking_s": round(t_host, 3), "n_b": int(bl["n_b"]), "n_c": int(bl["n_c"]),
            "ms_per_step": round(ms, 4), "iterations": it, "status": iccg.STATUS.get(st, st),
            "true_relres": float(np.linalg.norm(b - a.to_scipy() @ x) / np.linalg.norm(b)),
            "vs_parallel_leiden": {"ms_per_step": round(ms_par, 4), "iterations": it_par,
                                   "blocking_s": round(t_par, 3)}}


def ext_fp32(args, a, b, bl, x64, ms64, stream, dev):
    """Extension 1 on the same system and blocking: FP32 factors and
    substitutions, FP64 IC(0), CG scalars and x/r updates; same step."""
    import torch
    from paper_2609_00561_gb300 import iccg
    S = iccg.Solver(a, bl, precond_fp32=True, stream=stream.cuda_stream, factor=False)
    bd = torch.tensor(b, device=dev)
    xd = torch.zeros_like(bd)

    def step():
        iccg.iccg_factor(S.ctx)
        xd.zero_()
        return iccg.iccg_solve(S.ctx, bd, xd, args.tol, args.maxit, want_hist=False)

    for _ in range(max(1, args.warmup)):
        step()
    ms, (st, it, _) = time_steps(step, args.steps, stream)
    x = xd.cpu().numpy()
    S.close()
    return {"ms_per_step": round(ms, 4), "iterations": it, "status": iccg.STATUS.get(st, st),
            "true_relres": float(np.linalg.norm(b - a.to_scipy() @ x) / np.linalg.norm(b)),
            "rel_error_vs_fp64_gpu": float(np.linalg.norm(x - x64) / np.linalg.norm(x64)),
            "speedup_vs_fp64": round(ms64 / ms, 3), "_x": x}


def ext_batched(args, stream, dev, nsys=8, nrhs=16):
    """Extension 2, compact: 8 systems of config 4's recipe (sides U{16..64},
    shifts U[1e-4, 1e-1]) x 16 right-hand sides, ABMC 32, FP32 preconditioner,
    one launch; against the plain FP64 single-system solver run right-hand
    side by right-hand side."""
    import torch
    import oracle
    from paper_2609_00561_gb300 import iccg
    systems, _ = gen.config4(seed=args.seed, nsys=nsys, nrhs=nrhs)
    blocks = [iccg.blocking(a, "abmc", 32) for a, _ in systems]
    solvers = [iccg.Solver(a, bl, precond_fp32=True, lane_block_max=-1, stream=stream.cuda_stream)
               for (a, _), bl in zip(systems, blocks)]
    bs = iccg.BatchSolver(solvers, nrhs)
    B = [torch.tensor(b, device=dev) for _, b in systems]
    X = [torch.zeros_like(t) for t in B]
    bs.tune(B, args.tol, args.maxit)

    def step():
        for t in X:
            t.zero_()
        return bs.solve(B, X, args.tol, args.maxit)

    for _ in range(max(1, args.warmup)):
        step()
    ms, (st, its, stv, _) = time_steps(step, args.steps, stream)
    worst = 0.0
    for (a, b), t in zip(systems, X):
        m = a.to_scipy()
        xs = t.cpu().numpy()
        for j in range(nrhs):
            worst = max(worst, float(np.linalg.norm(b[j] - m @ xs[j]) / np.linalg.norm(b[j])))
    # the FP64 oracle on right-hand side 0 of the smallest system
    k0 = int(np.argmin([a.n for a, _ in systems]))
    a0, b0 = systems[k0]
    ref = oracle.iccg(a0, b0[0], blocks[k0]["perm"], tol=args.tol, maxit=args.maxit)
    x0 = X[k0].cpu().numpy()[0]
    err0 = float(np.linalg.norm(x0 - ref["x"]) / np.linalg.norm(ref["x"]))
    # plain FP64 single-system solver, right-hand side 0 of each system, x nrhs
    single = 0.0
    for (a, b), bl in zip(systems, blocks):
        S1 = iccg.Solver(a, bl, stream=stream.cuda_stream)
        bd = torch.tensor(b[0], device=dev)
        xd = torch.zeros_like(bd)
        iccg.iccg_solve(S1.ctx, bd, xd, args.tol, args.maxit, want_hist=False)

        def one():
            xd.zero_()
            return iccg.iccg_solve(S1.ctx, bd, xd, args.tol, args.maxit, want_hist=False)

        t1, _ = time_steps(one, 2, stream)
        single += t1
        S1.close()
    single *= nrhs
    shape = bs.info()
    bs.close()
    for S in solvers:
        S.close()
    return {"systems": nsys, "rhs_per_system": nrhs, "rows_total": int(sum(a.n for a, _ in systems)),
            "ms_per_step": round(ms, 4), "rhs_solves_per_s": round(nsys * nrhs / (ms * 1e-3), 1),
            "iterations": {"min": int(its.min()), "max": int(its.max())}, "status": iccg.STATUS.get(st, st),
            "worst_true_relres": worst, "rel_error_vs_fp64_oracle_rhs0_smallest": err0,
            "oracle_iterations": ref["iterations"], "gpu_iterations": int(its[k0, 0]),
            "plain_fp64_single_solves_ms": round(single, 3), "speedup_vs_plain_fp64": round(single / ms, 2),
            "shape": shape}


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
    """Extension 4: the learned blocking on the held-out matrices of the label
    sweep (config 5's recipe, n 1e5-2e6).  The model is selected and trained
    on the GPU with the library's kernels from the 160 training records; then
    every held-out matrix is solved live (FP64, to 1e-8) with the predicted
    ABMC block size and with the predicted CPM resolution, and, for
    comparison, with the best constant settings of the training labels and
    with the fixed settings of the paper's ranges (ABMC 32, CPM 0.05).  A step
    is the held-out set solved once with the predicted ABMC block size."""
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
    t0 = time.perf_counter()
    ens, rep = lm.report(data, seed=args.seed)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    cls, lg = ens.predict(X[te])
    gi = np.abs(lg[:, None] - np.log(np.array(gammas))[None, :]).argmin(axis=1)
    ia, ic = lm.best_constants(ta[tr], tc[tr])
    settings = ["abmc_predicted", "cpm_predicted", "abmc_best_constant", "cpm_best_constant", "abmc_fixed32",
                "cpm_fixed005"]
    times = {k: 0.0 for k in settings}
    per = []
    for k, idx in enumerate(te):
        spec = data["records"][idx]["spec"]
        a = gen.config5_matrix(spec)
        b = np.random.default_rng(spec["seed"] + 7).uniform(-1.0, 1.0, a.n)
        bd = torch.tensor(b, device=dev)
        want = {"abmc_predicted": ("abmc", bs_list[int(cls[k])]), "cpm_predicted": ("leiden_cpm", gammas[int(gi[k])]),
                "abmc_best_constant": ("abmc", bs_list[ia]), "cpm_best_constant": ("leiden_cpm", gammas[ic]),
                "abmc_fixed32": ("abmc", lm.BASE_BLOCK), "cpm_fixed005": ("leiden_cpm", lm.BASE_GAMMA)}
        done = {}
        row = {"index": int(spec["index"]), "kind": spec["kind"], "n": a.n}
        for name in settings:
            key = want[name]
            if key not in done:
                bl = iccg.blocking(a, key[0], key[1]) if key[0] == "abmc" else iccg.blocking(a, key[0], gamma=key[1])
                S = iccg.Solver(a, bl, stream=stream.cuda_stream)
                xd = torch.zeros_like(bd)
                iccg.iccg_solve(S.ctx, bd, xd, args.tol, args.maxit, want_hist=False)

                def one():
                    xd.zero_()
                    return iccg.iccg_solve(S.ctx, bd, xd, args.tol, args.maxit, want_hist=False)

                ms, _ = time_steps(one, max(1, args.steps), stream)
                S.close()
                done[key] = ms
            times[name] += done[key]
            row[name] = round(done[key], 3)
        per.append(row)
    result = {
        "metric": "ICCG time to 1e-8 rel. residual", "value": round(times["abmc_predicted"], 3), "unit": "ms",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(times["abmc_predicted"], 3),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS["learned"], "step": "the 40 held-out systems solved once each with the "
                   "predicted ABMC block size, inputs resident, blocking and setup excluded",
                   "l2": "mixed (systems of 1e5-2e6 rows)", "parallelism": "1 GPU"},
        "held_out_sum_ms": {k: round(v, 2) for k, v in times.items()},
        "gain_vs_fixed": {"abmc": round(times["abmc_fixed32"] / times["abmc_predicted"], 3),
                          "cpm": round(times["cpm_fixed005"] / times["cpm_predicted"], 3)},
        "gain_vs_best_constant": {"abmc": round(times["abmc_best_constant"] / times["abmc_predicted"], 3),
                                  "cpm": round(times["cpm_best_constant"] / times["cpm_predicted"], 3)},
        "selection_and_training_s": round(train_s, 2), "model_choice": rep["choice"],
        "held_out_vs_sweep": {"model": rep["test"], "best_constant": rep["test_best_constant"],
                              "fixed": rep["test_fixed"]},
        "per_matrix": per,
        "roofline": None, "e2e": None, "gpu_launches": None,
    }
    if rank == 0:
        print(json.dumps(result))


def oracle_solve(a, b, perm, args):
    """The oracle's full ICCG on the permuted system: IC(0), then PCG from
    x0 = 0 to the tolerance.  The permutation and lower-triangle extraction
    are setup (excluded like the GPU arm's).  Returns (IC(0) s, PCG s, x in
    the original numbering, iterations)."""
    import oracle
    perm = np.asarray(perm, dtype=np.int64)
    ah = oracle.permute(a, perm)
    lptr, lcol, aval = oracle.tril_csr(ah)
    bh = np.asarray(b)[perm]
    t0 = time.perf_counter()
    lval, _ = oracle.ic0(lptr, lcol, aval)
    t_ic = time.perf_counter() - t0
    t0 = time.perf_counter()
    xh, it, _, _ = oracle.pcg(ah, lptr, lcol, lval, bh, tol=args.tol, maxit=args.maxit)
    t_pcg = time.perf_counter() - t0
    x = np.zeros(a.n)
    x[perm] = xh
    return t_ic, t_pcg, x, it


def cpu_baseline(a, b, bl, args):
    t_ic, t_pcg, x, it = oracle_solve(a, b, bl["perm"], args)
    value_ms = (t_ic + t_pcg) * 1e3
    cb = {"value": round(value_ms, 1), "unit": "ms", "cores": 1, "kind": "oracle",
          "sample": f"one full solve of the same workload by the FP64 oracle (single thread): IC(0) "
                    f"{t_ic * 1e3:.0f} ms + PCG to {args.tol:g} in {it} iterations "
                    f"({t_pcg * 1e3 / max(it, 1):.1f} ms/iteration)"}
    return cb, x, it


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    # the reference arm never touches the GPU; blocking comes from the oracle
    # (bit-identical to the library's), each step is the oracle's full solve
    import oracle
    a, b = workload(args)
    bl = make_blocking(oracle, a, args)
    times, its = [], []
    for k in range(args.warmup + args.steps):
        t_ic, t_pcg, _, it = oracle_solve(a, b, bl["perm"], args)
        if k >= args.warmup:
            times.append(t_ic + t_pcg)
            its.append(it)
    ms = statistics.mean(times) * 1e3
    sample = (f"each step: one full solve by the FP64 oracle (single thread), IC(0) + PCG to {args.tol:g} "
              f"({its[-1]} iterations); permutation and blocking excluded as in the GPU arm")
    result = {"impl": "reference", "metric": "ICCG time to 1e-8 rel. residual", "value": round(ms, 1), "unit": "ms",
              "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 1),
              "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
              "dtype": "f32+f64" if args.fp32 else "f64", "data": "synthetic",
              "config": {"workload": workload_string(args, a, bl)},
              "iterations": its[-1],
              "cpu_baseline": {"value": round(ms, 1), "unit": "ms", "cores": 1, "kind": "oracle", "sample": sample},
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
    p.add_argument("--blocking", default=None,
                   choices=["abmc", "leiden_cpm", "leiden_md", "leiden_cpm_par", "leiden_md_par", "levels"],
                   help="default: leiden_cpm_par for poisson128, abmc otherwise")
    p.add_argument("--gamma", type=float, default=0.5, help="Leiden resolution (CPM threshold or modularity gamma)")
    p.add_argument("--split-levels", type=int, default=0,
                   help="split blocks above this many rows into in-block levels (0: no)")
    p.add_argument("--block-size", type=int, default=None, help="ABMC block size (default 8, or 32 for diffusion96)")
    p.add_argument("--tol", type=float, default=1e-8)
    p.add_argument("--maxit", type=int, default=5000)
    p.add_argument("--fp32", action="store_true", help="FP32 preconditioner (extension 1)")
    p.add_argument("--warps", type=int, default=0, help="warps per CTA of the substitution kernels (0: 8)")
    p.add_argument("--rows", type=int, default=0, help="rows per thread of a CTA group (0: 1)")
    p.add_argument("--lane-max", type=int, default=0,
                   help="largest block run as lane tiles (0: 32, -1: none, every color as CTA groups)")
    p.add_argument("--tile-mapping", default="auto", choices=["auto", "cta", "warp", "pair", "units"])
    p.add_argument("--fuse-sweep", type=int, default=0,
                   help="1: each preconditioner sweep as one cooperative launch (layouts of 1-2-row blocks)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-graph", action="store_true",
                   help="drive the PCG loop from the host (every kernel a separate launch, e.g. for ncu)")
    p.add_argument("--no-ext", action="store_true",
                   help="leave out the FP32-preconditioner and batched figures of the default line")
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
        args.blocking = "leiden_cpm_par" if args.workload == "poisson128" else "abmc"
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
