"""The N > 1 path of bench.py on the host: ranks as gloo processes on CPU
(world size 2).  bench.py runs one independent replica of the solve per GPU
("replicas only": a system does not shard), times each, and reports the
slowest replica's time; the reference arm runs on rank 0 only."""
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, loc = bench.dist_env()
    got = bench.max_over_ranks(10.0 + 5.0 * rank, torch.device("cpu"))
    out.put((r, w, loc, got))
    dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [(r, w, loc) for r, w, loc, _ in res] == [(0, 2, 0), (1, 2, 1)]
    assert all(got == 15.0 for *_, got in res)


def test_reference_arm_prints_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--nx", "16",
                        "--steps", "1", "--warmup", "0"],
                       capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
    env.update(RANK="0", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--nx", "16",
                        "--steps", "1", "--warmup", "0"],
                       capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "ms" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
    # the full workload (sizes, blocking, colors) as the GPU arm names it
    wl = line["config"]["workload"]
    assert "n=4096" in wl and "n_b=" in wl and "n_c=" in wl and "Leiden CPM resolution 0.5" in wl
    assert line["iterations"] > 0


def test_traffic_record_digest_ignores_comments_only():
    """The committed DRAM-traffic record is keyed by the kernel sources' code:
    a comment edit keeps the digest, any code edit changes it, and string
    literals (inline PTX) count as code."""
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    src = 'int a = 1;  // one\n/* block\n comment */\nasm("ld.global // not a comment");\n'
    assert bench.code_only(src) == 'int a = 1;\nasm("ld.global // not a comment");'
    assert bench.code_only(src.replace("// one", "// two\n// three")) == bench.code_only(src)
    assert bench.code_only(src.replace("a = 1", "a = 2")) != bench.code_only(src)
    assert bench.code_only(src.replace("// not a comment", "")) != bench.code_only(src)
