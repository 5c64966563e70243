"""Multi-rank path of the batched form, on the host: the LPT shard of a batch
is a balanced partition, and results computed rank by rank (here by the
float64 oracle, two gloo ranks on CPU) and gathered equal the single-process
results."""
import os
import socket

import numpy as np
import pytest

import oracle as O
from paper_2109_00626_gb300 import inputs as G
from paper_2109_00626_gb300 import shard as S
from paper_2109_00626_gb300 import workload as W

torch = pytest.importorskip("torch")


def _small_batch(n=14, seed=3):
    """Uneven batch in the shape of the 4096-pair workload, scaled down."""
    rng = np.random.default_rng(seed)
    out = []
    for p in range(n):
        order = int(rng.integers(2, 6))
        modes = [int(v) for v in rng.integers(2, 9, size=order)]
        rx = [1] + [int(v) for v in rng.integers(2, 12, size=order - 1)] + [1]
        ry = [1] + [int(v) for v in rng.integers(2, 12, size=order - 1)] + [1]
        out.append((modes, rx, ry, G.random_tt(rng, modes, rx), G.random_tt(rng, modes, ry)))
    return out


def test_lpt_shards_partition_and_balance():
    rng = np.random.default_rng(0)
    costs = list(rng.integers(1, 1000, size=257).astype(float))
    for world in (1, 2, 3, 8):
        shards = S.lpt_shards(costs, world)
        flat = sorted(i for s in shards for i in s)
        assert flat == list(range(len(costs)))
        loads = S.shard_loads(costs, shards)
        assert max(loads) <= sum(costs) / world + max(costs)
        assert shards == S.lpt_shards(costs, world)  # deterministic


def test_lpt_shards_of_the_4096_pair_workload():
    specs = G.batch4096_spec(4096)
    costs = [W.full_flops(s["modes"], s["ranks_x"], s["ranks_y"]) if s["kind"] == "full"
             else W.partial_chain_flops(s["modes"], s["ranks_x"], s["ranks_y"], s["mask"]) for s in specs]
    for world in (2, 4, 8):
        loads = S.shard_loads(costs, S.lpt_shards(costs, world))
        assert max(loads) / (sum(costs) / world) < 1.01


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _gloo_worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        batch = _small_batch()
        costs = [W.full_flops(m, rx, ry) for m, rx, ry, _, _ in batch]
        mine = S.lpt_shards(costs, world)[rank]
        vals = [O.contract_full(batch[p][3], batch[p][4]) for p in mine]
        full = S.gather_values(mine, vals, len(batch)).numpy()
        slowest = S.max_over_ranks(float(rank) + 0.5)
        q.put((rank, full.tolist(), slowest, len(mine)))
    finally:
        dist.destroy_process_group()


def test_sharded_batch_gloo_two_ranks():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_gloo_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    batch = _small_batch()
    want = [O.contract_full(x, y) for _, _, _, x, y in batch]
    assert sum(n for _, _, _, n in got) == len(batch)
    for rank, full, slowest, _ in got:
        np.testing.assert_allclose(full, want, rtol=0, atol=0)  # each value computed once, by one rank
        assert slowest == 1.5
