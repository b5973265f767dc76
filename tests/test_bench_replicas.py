"""The N > 1 bench path on CPU: two gloo ranks run the replica plumbing of
bench.py (barrier, max over ranks, whole-job value) and the reference arm
prints only on rank 0."""
import contextlib
import io
import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    ranks = bench.Ranks("gloo", "cpu")
    ranks.barrier()
    slowest = ranks.max(1.0 + rank)             # rank r "took" 1 + r seconds
    value = bench.replica_value(1000.0, 4, slowest, ranks.world)
    ranks.barrier()
    ranks.close()
    out.put((rank, ranks.world, slowest, value))


def test_two_gloo_ranks_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, world, slowest, value in res:
        assert world == 2
        assert slowest == 2.0                   # max over ranks
        assert value == 2 * 1000.0 * 4 / 2.0    # all ranks' units / slowest time


def test_single_process_needs_no_process_group(monkeypatch):
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    sys.path.insert(0, ROOT)
    import bench
    r = bench.Ranks("gloo", "cpu")
    assert (r.world, r.rank) == (1, 0) and r.dist is None
    assert r.max(3.5) == 3.5
    r.close()


def test_reference_arm_is_silent_on_other_ranks(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    called = []
    monkeypatch.setattr(bench, "run_oracle", lambda **kw: called.append(kw))
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.reference_arm(type("A", (), {"steps": 2, "warmup": 1})())
    assert buf.getvalue() == "" and called == []


def test_all_cores_oracle_leg_counts_every_process():
    """The all-cores CPU leg runs one single-threaded oracle process per core
    and reports their summed work over the slowest process's time."""
    sys.path.insert(0, ROOT)
    import bench
    r = bench.run_oracle_all_cores(nsamp=2, budget=0.2)
    assert r["kind"] == "oracle" and r["cores"] >= 1 and r["value"] > 0
    assert f"{r['cores']} processes" in r["sample"]
