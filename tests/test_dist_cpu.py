"""The N > 1 plumbing of bench.py on CPU: two gloo ranks, barrier and max over ranks, and the
whole-job throughput formula (units all ranks processed / max time)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    d = bench.Dist("gloo")
    d.barrier()
    t = d.max(10.0 + rank)  # rank r "took" 10 + r ms
    v = bench.whole_job_rate(1000, 5, d.world, t)
    out.put((rank, d.world, t, v))
    d.barrier()
    d.close()


def test_two_gloo_ranks_max_and_rate():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, world, t, v in res:
        assert world == 2 and t == 11.0
        # 1000 updates x 5 steps on each of 2 ranks in the slowest rank's 11 ms
        assert v == pytest.approx(1000 * 5 * 2 / 0.011)


def test_single_process_defaults():
    sys.path.insert(0, ROOT)
    import bench
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        os.environ.pop(k, None)
    d = bench.Dist("gloo")
    assert d.world == 1 and d.rank == 0 and d.max(3.5) == 3.5
    assert bench.whole_job_rate(10, 2, 1, 4.0) == pytest.approx(10 * 2 / 0.004)


def test_traffic_key_ignores_comments():
    """The DRAM-traffic figure is keyed by the forward kernel's code with comments and
    whitespace removed: a comment edit keeps the key, a code edit changes it."""
    import bench
    src = 'int a = 1; // one\n/* block\n comment */ const char *s = "// not a comment";\n'
    assert bench.code_only(src) == bench.code_only('int a = 1;\nconst char *s = "// not a comment";')
    assert bench.code_only(src) != bench.code_only(src.replace("a = 1", "a = 2"))
    assert '"//notacomment"' in bench.code_only(src)
    key = bench.kernel_source_hash()
    assert len(key) == 12 and key == bench.kernel_source_hash()
