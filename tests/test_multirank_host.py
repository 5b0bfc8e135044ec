"""Host logic of bench.py's multi-rank paths, on CPU with the gloo backend.

Two processes form a process group on 127.0.0.1.  The batched workload is
sharded over the ranks with no data-path exchange: the shards must be disjoint
and cover every instance.  The whole-job figures are a sum of the ranks' work
over the slowest rank's time.
"""
import importlib.util
import os
import socket

import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")
mp = pytest.importorskip("torch.multiprocessing")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import sys
    sys.path.insert(0, ROOT)
    import workloads as W
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench = _bench()
    inst = W.batched_instances(37)
    mine = bench.shard(inst, rank, world)
    dofs = sum(w.n_dofs for w in mine)
    t = 1.0 + rank                      # the slower rank sets the job time
    tmax = bench.reduce_across_ranks(t, "max", dist)
    dofs_all = bench.reduce_across_ranks(dofs, "sum", dist)
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write(f"{tmax} {dofs_all} {','.join(w.name for w in mine)}\n")
    dist.barrier()
    dist.destroy_process_group()


def test_batched_sharding_and_reductions_two_ranks(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    import sys
    sys.path.insert(0, ROOT)
    import workloads as W
    inst = W.batched_instances(37)
    names = []
    for r in range(world):
        tmax, dofs_all, shard_names = open(tmp_path / f"rank{r}.txt").read().split()
        assert float(tmax) == 2.0
        assert int(float(dofs_all)) == sum(w.n_dofs for w in inst)
        names += shard_names.split(",")
    assert sorted(names) == sorted(w.name for w in inst)
    assert len(set(names)) == len(names)


def test_single_process_reduction_is_identity():
    bench = _bench()
    assert bench.reduce_across_ranks(3.5, "max", None) == 3.5
    assert bench.shard(range(5), 0, 1) == [0, 1, 2, 3, 4]
