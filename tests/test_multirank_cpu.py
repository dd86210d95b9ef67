"""The N>1 host logic of bench.py on CPU with two gloo ranks: the
max-over-ranks timing, the whole-job throughput, and the sharding of
independent graphs (the batching workload) across ranks. The V-cycle of
one hypergraph does not shard (replicas only), so no data-path collective
exists to test."""

import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    import json
    import bench
    import hypergen
    import torch.distributed as dist
    bench.init_dist(ws, "gloo")
    # every rank measured a different time: the job's time is the slowest
    t = bench.max_over_ranks(1.0 + rank, ws)
    bench.barrier(ws)
    specs = hypergen.batch_specs(256)
    weights = [sp.n for sp in specs]
    mine = bench.shard_units(weights, ws, rank)
    load = float(sum(weights[i] for i in mine))
    tot = bench.max_over_ranks(load, ws)
    json.dump({"max_t": t, "mine": mine, "load": load, "max_load": tot,
               "agg": bench.aggregate(100.0, [t] * ws)},
              open(os.path.join(out_dir, "r%d.json" % rank), "w"))
    dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    import json
    import torch.multiprocessing as mp
    ws = 2
    mp.start_processes(_worker, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, join=True,
                       start_method="spawn")
    r = [json.load(open(tmp_path / ("r%d.json" % i))) for i in range(ws)]
    assert r[0]["max_t"] == r[1]["max_t"] == 2.0
    assert r[0]["agg"] == pytest.approx(100.0 * ws / 2.0)
    every = sorted(r[0]["mine"] + r[1]["mine"])
    assert every == list(range(256))                       # each graph exactly once
    assert abs(r[0]["load"] - r[1]["load"]) <= 0.01 * (r[0]["load"] + r[1]["load"])


def test_shard_units_is_balanced_and_complete():
    sys.path.insert(0, ROOT)
    import bench
    w = [5, 1, 1, 1, 1, 1, 3, 3]
    for ws in (1, 2, 3, 8):
        parts = [bench.shard_units(w, ws, r) for r in range(ws)]
        assert sorted(i for p in parts for i in p) == list(range(len(w)))
        loads = [sum(w[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(w)


def _spawned_payload(argv):
    """What each rank runs in the spawn test: the environment torchrun would
    set, a gloo group, and the max-over-ranks timing of bench.py."""
    sys.path.insert(0, ROOT)
    import json
    import bench
    import torch.distributed as dist
    ws, rank, local = bench.dist_env()
    bench.init_dist(ws, "gloo")
    t = bench.max_over_ranks(0.5 * (rank + 1), ws)
    json.dump({"ws": ws, "rank": rank, "local": local, "t": t,
               "addr": os.environ["MASTER_ADDR"], "argv": argv},
              open(os.path.join(argv[0], "s%d.json" % rank), "w"))
    dist.destroy_process_group()


def test_spawn_ranks_sets_the_launcher_environment(tmp_path):
    """bench.py --gpus N without torchrun starts N ranks itself through
    spawn_ranks; each sees RANK / LOCAL_RANK / WORLD_SIZE and 127.0.0.1."""
    import json
    sys.path.insert(0, ROOT)
    import bench
    bench.spawn_ranks(3, _spawned_payload, [str(tmp_path)])
    r = [json.load(open(tmp_path / ("s%d.json" % i))) for i in range(3)]
    assert [x["rank"] for x in r] == [0, 1, 2] and [x["local"] for x in r] == [0, 1, 2]
    assert all(x["ws"] == 3 and x["t"] == 1.5 and x["addr"] == "127.0.0.1" for x in r)


def test_gpus_flag_must_match_the_launcher(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "0")
    with pytest.raises(SystemExit):
        bench.main(["--gpus", "4", "--workload", "small_2k"])
    with pytest.raises(SystemExit):
        bench.main(["--gpus", "0"])
