"""Host logic of bench.py on the CPU.  N > 1: two gloo ranks (127.0.0.1) reduce their timings
to the maximum over ranks, the whole-job throughput of independent replicas is all ranks' work
over the slowest rank's time, and the reference arm does nothing on ranks other than 0 (the
apply itself does not shard -- replicas only -- so these are the only multi-rank steps).
Roofline: the kernel code hash behind the traffic reference ignores comments."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        mx = bench.max_over_ranks([1.5 + rank, 10.0 - rank, 0.25 * (rank + 1)], "cpu")
        out.put((rank, mx))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    world, port = 2, _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(world):
        assert got[r] == [2.5, 10.0, 0.5]


def test_replica_throughput_and_single_process_identity():
    sys.path.insert(0, ROOT)
    import bench
    # one process: the reduction is the identity
    assert bench.max_over_ranks([3.0, 4.0], "cpu") == [3.0, 4.0]
    # 4 replicas of 2M unknowns x 20 steps, slowest replica 0.5 s
    assert bench.replica_throughput(4, 2_097_152, 20, 0.5) == 4 * 2_097_152 * 20 / 0.5


def test_reference_arm_is_rank0_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")

    class A:
        steps, warmup, gpus, tol, precision = 5, 3, 2, 0.0, "mixed"

    assert bench.run_reference(A()) is None
    assert capsys.readouterr().out == ""


def test_code_hash_ignores_comments_only(tmp_path):
    """The roofline traffic reference stays valid across comment edits of the kernel source and
    becomes invalid when code changes."""
    sys.path.insert(0, ROOT)
    import bench
    a = tmp_path / "a.cu"
    b = tmp_path / "b.cu"
    c = tmp_path / "c.cu"
    a.write_text('// header\nint f(int x) {\n  return x + 1;  // add one\n}\n\nconst char* s = "a // b";\n')
    b.write_text('// other header\n\nint f(int x) {\n  return x + 1;\n}\nconst char* s = "a // b";\n')
    c.write_text('// header\nint f(int x) {\n  return x + 2;  // add one\n}\n\nconst char* s = "a // b";\n')
    assert bench.code_hash(str(a)) == bench.code_hash(str(b))
    assert bench.code_hash(str(a)) != bench.code_hash(str(c))
