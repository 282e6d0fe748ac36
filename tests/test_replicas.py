"""Host-side logic of the multi-process (one process per GPU) layout, on CPU:
instance sharding and the max-over-ranks reduction, with world_size-2 gloo
process groups on 127.0.0.1."""
import os
import socket

import pytest

import lbm_inputs as I

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")

from paper_2107_06355_gb300.replicas import max_over_ranks, shard_instances  # noqa: E402


def test_shards_cover_every_instance_once_and_balance_nodes():
    specs = I.batch_specs()
    sizes = [s["nx"] * s["ny"] for s in specs]
    for ws in (1, 2, 3, 4, 8):
        shards = shard_instances(sizes, ws)
        flat = sorted(i for s in shards for i in s)
        assert flat == list(range(len(sizes)))
        loads = [sum(sizes[i] for i in s) for s in shards]
        # longest-processing-time: no rank exceeds the mean by more than the largest instance
        assert max(loads) <= sum(sizes) / ws + max(sizes)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, sizes, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = shard_instances(sizes, world)[rank]
    # each rank "times" its shard: here its node count stands in for a duration
    local = float(sum(sizes[i] for i in mine))
    mx = max_over_ranks(local)
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as fh:
        fh.write(f"{mx} {local} {sorted(i for g in gathered for i in g)}\n")
    dist.destroy_process_group()


def test_two_rank_gloo_shards_and_max_reduction(tmp_path):
    import torch.multiprocessing as mp

    sizes = [s["nx"] * s["ny"] for s in I.batch_specs()]
    mp.spawn(_worker, args=(2, _free_port(), sizes, str(tmp_path)), nprocs=2, join=True)
    lines = [open(tmp_path / f"r{r}.txt").read().split(" ", 2) for r in range(2)]
    mxs = {float(l[0]) for l in lines}
    locals_ = [float(l[1]) for l in lines]
    assert mxs == {max(locals_)}
    assert sum(locals_) == float(sum(sizes))
    for l in lines:
        assert l[2].strip() == str(list(range(len(sizes))))

