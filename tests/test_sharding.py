"""Host logic of the multi-GPU batch: the assignment of independent meshes to
ranks (greedy longest-processing-time rule), single-process properties and a
world-size-2 gloo run in which each rank computes its share independently."""
import os
import socket

import pytest

from paper_2103_14870_gb300.sharding import assign_meshes


def test_assignment_is_a_partition_and_balanced():
    sizes = [7, 3, 9, 9, 1, 4, 4, 12, 0, 5]
    for world in (1, 2, 3, 4, 16):
        parts = assign_meshes(sizes, world)
        assert len(parts) == world
        flat = sorted(k for p in parts for k in p)
        assert flat == list(range(len(sizes)))
        loads = [sum(sizes[k] for k in p) for p in parts]
        # LPT: the largest load exceeds the mean by at most the largest item
        assert max(loads) <= sum(sizes) / world + max(sizes)
    assert assign_meshes(sizes, 1) == [list(range(len(sizes)))]


def test_assignment_known_case_and_errors():
    # 8, 7, 6, 5, 4 over 2 ranks: 8 -> r0, 7 -> r1, 6 -> r1 (7 < 8), 5 -> r0 (8 < 13), 4 -> r0 (13 = 13: lower rank)
    assert assign_meshes([8, 7, 6, 5, 4], 2) == [[0, 3, 4], [1, 2]]
    with pytest.raises(ValueError):
        assign_meshes([1, 2], 0)
    with pytest.raises(ValueError):
        assign_meshes([1, -2], 2)


def test_batch_configuration_shards_evenly():
    from workloads import batch_configs
    sizes = [w.n_tets for w in batch_configs()]
    for world in (2, 4, 8):
        loads = [sum(sizes[k] for k in p) for p in assign_meshes(sizes, world)]
        assert max(loads) <= 1.10 * sum(sizes) / world + 1   # within 10% of an even split


def _worker(rank, world, port, sizes, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = assign_meshes(sizes, world)[rank]
    got = [None] * world
    dist.all_gather_object(got, mine)
    q.put((rank, mine, got))
    dist.destroy_process_group()


def test_two_rank_gloo_shares_agree():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    sizes = [5000, 80000, 12000, 2000, 40000, 33000, 7000]
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, sizes, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, mine0, got0), (r1, mine1, got1) = res
    assert got0 == got1 == [mine0, mine1]
    assert sorted(mine0 + mine1) == list(range(len(sizes)))
    assert not set(mine0) & set(mine1)
