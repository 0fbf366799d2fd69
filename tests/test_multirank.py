"""The benchmark's host logic on CPU.  Multi-rank (gloo, world size 2): every
rank runs its own replica of the sequence (no collective on the data path);
the job's time is the slowest rank's (an all-reduce MAX of the per-rank
times) and its throughput counts every rank's solves; the reference arm's
work runs on rank 0 only.  The reference (oracle) arm's JSON line."""
import multiprocessing as mp
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(times[rank], dist, "cpu")
        dist.barrier()
        out.put((rank, ms, bench.job_throughput(80, 2, world, ms)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_throughput_with_gloo():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    world, port = 2, _free_port()
    times = [1200.0, 1500.0]   # ms per rank: rank 1 is the slower one
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, times, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in res:
        assert ms == 1500.0                              # every rank sees the slowest time
        assert abs(value - 80 * 2 * 2 / 1.5) < 1e-9      # all ranks' solves over that time


def test_single_process_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert abs(bench.job_throughput(80, 2, 1, 3000.0) - 80 * 2 / 3.0) < 1e-12


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    """A rank other than 0 returns without timing anything."""
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setattr(bench, "cpu_oracle_timing", lambda *a, **k: (_ for _ in ()).throw(AssertionError("ran")))
    args = bench.argparse.Namespace(quick=True, warmup=3, steps=1, shifts=20, k=20, rhs=4, gpus=2, N=48)
    assert bench.run_reference(args) is None


def test_reference_arm_line_on_cpu():
    """The oracle arm prints the contract's line on the workload config the
    GPU arm names (small grid: a few seconds of oracle work)."""
    import json
    import subprocess
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--quick",
                          "--steps", "1", "--warmup", "3"], capture_output=True, text=True, timeout=600,
                         env=dict(os.environ, RANK="0", WORLD_SIZE="1"))
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    sys.path.insert(0, ROOT)
    import bench
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == "solves/s"
    assert line["higher_is_better"] is True and line["value"] > 0 and line["steps"] == 1 and line["warmup"] == 3
    cfg = line["config"]
    assert cfg["workload"] == "3d-7pt-conv-diff-48^3-shifted"
    assert cfg["n"] == 48 ** 3 and cfg["nnz"] == 7 * 48 ** 3 - 6 * 48 ** 2   # 7-point stencil, Dirichlet boundary
    assert cfg["k"] == 20 and cfg["tol"] == 1e-8 and cfg["cycle_s"] == 25
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "solves/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
