"""The multi-rank path of bench.py on CPU: two gloo ranks, each with its own
system seeds, a barrier, the maximum over ranks of the timed seconds and the
whole-job throughput."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    os.environ.update({"WORLD_SIZE": str(ws), "RANK": str(rank), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    from paper_2510_21213_gb300 import dist as pd

    ws_, rank_, _ = pd.init("gloo")
    seeds = pd.rank_seeds(4000, 3, rank_)
    pd.barrier(sync_cuda=False)
    seconds = 1.5 + rank_  # rank 1 is the slow one
    tmax = pd.max_over_ranks(seconds)
    rate = pd.aggregate_rate(10, 2, tmax, ws_)
    out[rank_] = (ws_, seeds, tmax, rate)
    pd.finish()


def test_two_gloo_ranks():
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_worker, args=(2, port, out), nprocs=2, start_method="spawn")
        res = dict(out)
    assert set(res) == {0, 1}
    for r in (0, 1):
        ws, seeds, tmax, rate = res[r]
        assert ws == 2
        assert tmax == 2.5  # the maximum, seen by both ranks
        assert rate == pytest.approx(2 * 10 * 2 / 2.5)
    assert set(res[0][1]).isdisjoint(res[1][1])  # every rank builds its own systems


def test_single_rank_defaults(monkeypatch):
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    from paper_2510_21213_gb300 import dist as pd

    assert pd.env() == (1, 0, 0)
    assert pd.max_over_ranks(3.0) == 3.0
    assert pd.rank_seed(2, 0) == 2
    with pytest.raises(ValueError):
        pd.aggregate_rate(1, 1, 0.0, 1)
