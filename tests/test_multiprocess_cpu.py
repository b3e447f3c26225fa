"""The N > 1 host logic of bench.py on the CPU, with world_size-2 gloo process
groups: the barrier and the max-over-ranks reduction of the timing (the
replicas-only multi-GPU mode), and the reference arm's rule that only rank 0
works and prints."""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        bench.barrier(world)
        # per-rank step times: the job's time is the slowest rank's
        got = bench.max_over_ranks(10.0 + 5.0 * rank, world)
        bench.barrier(world)
        out.put((rank, got))
    finally:
        dist.destroy_process_group()


def test_barrier_and_max_over_ranks_gloo():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = dict(q.get(timeout=10) for _ in range(world))
    assert got == {0: 15.0, 1: 15.0}


def test_max_over_ranks_is_identity_at_one_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, 1) == 3.25


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "3"],
                       capture_output=True, text=True, timeout=120, env=env, cwd=ROOT)
    assert r.returncode == 0 and r.stdout.strip() == "", r.stdout + r.stderr


def test_stopping_study_rows():
    """bench.py's stopping-study rows from a check trace: relative residual,
    the certified bound gap/(f - gap) (None while f <= gap) and the true
    relative error against f*; at most `keep` rows, first and last kept."""
    sys.path.insert(0, ROOT)
    import bench
    tr = [{"h": 16 * i, "res": 2.0 ** -i, "gap": 4.0 ** -i, "fval": 1.0 + 2.0 ** -i}
          for i in range(100)]
    tr[0]["gap"] = 5.0  # gap above f: no certificate yet
    rows = bench._trajectory(tr, 1.0, keep=10)
    assert len(rows) == 10 and rows[0]["h"] == 0 and rows[-1]["h"] == 16 * 99
    assert rows[0]["rel_residual"] == 1.0 and rows[0]["certified_rel_obj_err"] is None
    r = rows[5]
    i = r["h"] // 16
    assert abs(r["certified_rel_obj_err"] - 4.0 ** -i / (1.0 + 2.0 ** -i - 4.0 ** -i)) < 1e-15
    assert abs(r["true_rel_obj_err"] - 2.0 ** -i) < 1e-15
    assert all(x["true_rel_obj_err"] is None for x in bench._trajectory(tr, None, keep=5))
