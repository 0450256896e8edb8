"""Host logic of the multi-GPU replica mode on CPU: world_size-2 gloo process groups.

The replicas exchange nothing on the data path; what crosses ranks is the
benchmark's (max time, summed work) pair and the weighted orientation average
of results solved on different ranks.  Both are checked here against the
single-process computation, with each rank holding only its own share.
"""
import os
import socket
import tempfile

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1002_1505_gb300 import replicas  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _library_built():
    # the weighted orientation sum runs in the C-ABI library (host-only entry point)
    from paper_1002_1505_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()


@pytest.mark.parametrize("world", [1, 2, 3, 4, 7])
def test_shard_covers_every_orientation_once(world):
    for n in range(0, 40):
        seen = []
        sizes = []
        for rank in range(world):
            a, b = replicas.shard(n, rank, world)
            assert 0 <= a <= b <= n
            seen.extend(range(a, b))
            sizes.append(b - a)
        assert seen == list(range(n))  # contiguous, in rank order, each exactly once
        assert max(sizes) - min(sizes) <= 1


def test_shard_rejects_bad_ranks():
    with pytest.raises(ValueError):
        replicas.shard(4, 2, 2)
    with pytest.raises(ValueError):
        replicas.shard(-1, 0, 1)


def test_single_process_reductions_are_local():
    assert replicas.reduce_max_sum(3.5, 7.0) == (3.5, 7.0)
    q = np.arange(12.0).reshape(6, 2)
    w = np.array([0.2, 0.3, 0.5])
    np.testing.assert_allclose(replicas.orientation_average_sharded(q, w, iorth=2),
                               np.tensordot(w, q.reshape(3, 2, 2), axes=(0, 0)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


N_ORI, IORTH, NQ = 7, 2, 4


def _problem():
    rng = np.random.default_rng(11)
    q = rng.normal(size=(N_ORI * IORTH, NQ))  # per-RHS results, orientation-major
    w = rng.uniform(0.5, 1.5, size=N_ORI)
    return q, w / w.sum()


def _rank_main(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q, w = _problem()
        a, b = replicas.shard(N_ORI, rank, world)
        avg = replicas.orientation_average_sharded(q[a * IORTH:b * IORTH], w[a:b], iorth=IORTH)
        t, u = replicas.reduce_max_sum(10.0 + rank, float(b - a))
        np.save(os.path.join(out_dir, f"avg{rank}.npy"), avg)
        np.save(os.path.join(out_dir, f"tu{rank}.npy"), np.array([t, u]))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_reduce_like_one_process(world):
    q, w = _problem()
    ref = np.tensordot(w, q.reshape(N_ORI, IORTH, NQ), axes=(0, 0))
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_rank_main, args=(world, _free_port(), d), nprocs=world, join=True,
                           start_method="spawn")
        for rank in range(world):
            np.testing.assert_allclose(np.load(os.path.join(d, f"avg{rank}.npy")), ref, rtol=1e-14, atol=1e-15)
            t, u = np.load(os.path.join(d, f"tu{rank}.npy"))
            assert t == 10.0 + (world - 1)  # slowest rank
            assert u == N_ORI              # every orientation counted once
