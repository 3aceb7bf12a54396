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


def test_shard_range_covers_and_balances():
    from paper_2510_21213_gb300 import dist as pd

    for n in (0, 1, 4, 56, 2081):
        for ws in (1, 2, 3, 8):
            parts = [pd.shard_range(n, ws, r) for r in range(ws)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            assert all(parts[r][1] == parts[r + 1][0] for r in range(ws - 1))
            sizes = [e - b for b, e in parts]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        pd.shard_range(10, 2, 2)


def _sharded_worker(rank, ws, port, out):
    os.environ.update({"WORLD_SIZE": str(ws), "RANK": str(rank), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import numpy as np

    import oracle
    from paper_2510_21213_gb300 import dist as pd
    from paper_2510_21213_gb300 import inputs

    ws_, rank_, _ = pd.init("gloo")
    spec = inputs.tiny_system()
    m = oracle.Mesh(spec.mesh.lo, spec.mesh.hi, spec.mesh.n, spec.mesh.p)
    psi = inputs.orbitals(spec, oracle.node_coords(m), oracle.quad_weights(m))
    K, eh, ex = pd.sharded_exchange(lambda b, e: oracle.exchange_partial(m, psi, b, e), psi.shape[0], ws_, rank_)
    out[rank_] = (np.asarray(K).tolist(), eh, ex)
    pd.finish()


def test_sharded_exchange_on_two_gloo_ranks():
    """One system's exchange build split over two CPU ranks (each computes its
    share of the sources with the oracle) and reduced by all-reduce: the same
    K, E_H and E_X as the whole build."""
    import numpy as np

    import oracle
    from paper_2510_21213_gb300 import inputs

    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_sharded_worker, args=(2, port, out), nprocs=2, start_method="spawn")
        res = dict(out)
    spec = inputs.tiny_system()
    m = oracle.Mesh(spec.mesh.lo, spec.mesh.hi, spec.mesh.n, spec.mesh.p)
    psi = inputs.orbitals(spec, oracle.node_coords(m), oracle.quad_weights(m))
    ref = oracle.exchange_build(m, psi)
    for r in (0, 1):
        K, eh, ex = res[r]
        K = np.asarray(K)
        assert np.abs(K - ref["K"]).max() <= 1e-12 * np.abs(ref["K"]).max()
        assert abs(eh - ref["E_H"]) <= 1e-12 * abs(ref["E_H"])
        assert abs(ex - ref["E_X"]) <= 1e-12 * abs(ref["E_X"])
