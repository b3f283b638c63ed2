"""Label sweep for the learned blocking: for every matrix of the generated set,
the FP64 GPU ICCG solve time to 1e-8 under ABMC blocking with each block size
of BLOCK_SIZES and under Leiden CPM blocking with each resolution of GAMMAS
(greedy block coloring in both cases).  Blockings run in a process pool on
the host (production C++ blocking, no GPU); solves run in the main process.

    python -m paper_2609_00561_gb300.learn.sweep --out blocking_sweep.json \
        [--count 200] [--n-lo 2e4] [--n-hi 2e5] [--workers 12]
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# the paper's ranges (block sizes 8..128, resolutions 0.01..0.5) extended on
# both sides: on GB300 the fastest settings lie at or beyond their small-block
# ends (block size 8 and resolution 0.5 won on every matrix of a first sweep)
BLOCK_SIZES = [2, 4, 8, 16, 32, 64, 128]
GAMMAS = [0.01, 0.02, 0.05, 0.1, 0.2, 0.5, 1.0, 2.0]


def _blockings(spec):
    import numpy as np  # noqa: F401
    import gen
    from paper_2609_00561_gb300 import iccg
    a = gen.config5_matrix(spec)
    out = []
    for s in BLOCK_SIZES:
        t0 = time.perf_counter()
        bl = iccg.blocking(a, "abmc", s)
        out.append(("abmc", s, bl, time.perf_counter() - t0))
    for g in GAMMAS:
        t0 = time.perf_counter()
        bl = iccg.blocking(a, "leiden_cpm", gamma=g)
        out.append(("leiden_cpm", g, bl, time.perf_counter() - t0))
    return spec, a, out


def _time_solve(a, bl, b, tol, maxit, reps):
    import torch
    from paper_2609_00561_gb300 import iccg
    S = iccg.Solver(a, bl)
    bd = torch.tensor(b, device="cuda")
    xd = torch.zeros_like(bd)
    st, it, _ = iccg.iccg_solve(S.ctx, bd, xd, tol, maxit, want_hist=False)
    best = float("inf")
    for _ in range(reps):
        xd.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        st, it, _ = iccg.iccg_solve(S.ctx, bd, xd, tol, maxit, want_hist=False)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    info = S.info()
    S.close()
    return best, int(it), int(st), info


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--out", required=True)
    p.add_argument("--count", type=int, default=200)
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--n-lo", type=float, default=2e4)
    p.add_argument("--n-hi", type=float, default=2e5)
    p.add_argument("--workers", type=int, default=12)
    p.add_argument("--tol", type=float, default=1e-8)
    p.add_argument("--maxit", type=int, default=20000)
    p.add_argument("--reps", type=int, default=2)
    args = p.parse_args()
    import gen
    from paper_2609_00561_gb300 import build
    build.build()
    specs = gen.config5_specs(args.count, seed=args.seed, n_lo=args.n_lo, n_hi=args.n_hi)
    ctx = mp.get_context("spawn")     # the pool starts before any GPU call
    records = []
    t_start = time.perf_counter()
    with ctx.Pool(args.workers) as pool:
        import numpy as np
        for k, (spec, a, bls) in enumerate(pool.imap(_blockings, specs)):
            b = np.random.default_rng(spec["seed"] + 7).uniform(-1.0, 1.0, a.n)
            runs = []
            for method, param, bl, tb in bls:
                ms, it, st, info = _time_solve(a, bl, b, args.tol, args.maxit, args.reps)
                runs.append({"method": method, "param": param, "ms": ms, "iterations": it, "status": st,
                             "n_b": int(bl["n_b"]), "n_c": int(bl["n_c"]), "blocking_s": tb,
                             "tile_colors": info["tile_colors"]})
            records.append({"spec": spec, "n": a.n, "nnz": a.nnz, "runs": runs})
            print(f"[{k + 1}/{len(specs)}] {spec['kind']} n={a.n} "
                  f"best abmc {min(r['ms'] for r in runs[:5]):.1f} ms "
                  f"best cpm {min(r['ms'] for r in runs[5:]):.1f} ms "
                  f"({time.perf_counter() - t_start:.0f} s)", flush=True)
    meta = {"block_sizes": BLOCK_SIZES, "gammas": GAMMAS, "tol": args.tol, "seed": args.seed,
            "n_lo": args.n_lo, "n_hi": args.n_hi, "count": args.count,
            "timing": "FP64 iccg_solve, CUDA events, best of reps after one untimed solve",
            "rhs": "U[-1,1], numpy default_rng(spec seed + 7)"}
    with open(args.out, "w") as f:
        json.dump({"meta": meta, "records": records}, f)


if __name__ == "__main__":
    main()
