"""The multi-GPU mode is replicas only: each rank renders its own views, and the only exchange is
the max-reduce of the timed region's length.  This checks bench.py's host logic for it with two
gloo ranks on the CPU (no GPU): the ranks start on different views and together cover every
camera, every rank sees the slowest rank's time, and the whole-job rate counts every rank's
pixels."""
import importlib.util
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        b = _bench()
        assert b._dist() == (ws, rank, rank)
        cams = list(range(20))
        mine = b.replica_cameras(cams, rank)
        ms = b.max_over_ranks(10.0 * (rank + 1), dist, "cpu")  # rank r took 10 (r + 1) ms
        rate = b.aggregate_mpix_s(ws, 1_000_000, 5, ms)
        out[rank] = (mine, ms, rate)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_replicas():
    ws = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    assert set(res) == {0, 1}
    cams0, ms0, rate0 = res[0]
    cams1, ms1, rate1 = res[1]
    assert sorted(cams0) == sorted(cams1) == list(range(20))  # each rank cycles through every view
    assert cams0[0] != cams1[0]                               # starting on different views
    assert ms0 == ms1 == 20.0                                 # the slowest rank's time, everywhere
    assert rate0 == rate1 == pytest.approx(ws * 1_000_000 * 5 / 0.020 / 1e6)


def test_single_process_needs_no_group():
    b = _bench()
    assert b.max_over_ranks(7.5, None, "cpu") == 7.5
    assert b.replica_cameras([1, 2, 3], 0) == [1, 2, 3]
    assert b.aggregate_mpix_s(1, 1_000_000, 10, 100.0) == pytest.approx(100.0)
