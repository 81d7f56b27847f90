"""Host logic of the multi-rank benchmark (bench.py under torchrun), run as
two gloo ranks on the CPU: each rank builds its own seeded share of the
sweep (weak scaling: the capillaries differ between ranks, their
distributions do not), and the line rank 0 prints takes the slowest
rank's time and the fluid nodes of all ranks.  The batch has no exchange
step, so no collective touches the data path."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as td
    td.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port,
                          rank=rank, world_size=world)
    import bench
    geoms, params, desc = bench.build_workload("sweep", rank, lattices=3)
    n = bench.fluid_nodes(geoms)
    widths = [g.solid.shape[0] for g in geoms]
    ms, total = bench.combine_ranks(10.0 * (rank + 1), n, "cpu")
    import json
    with open(os.path.join(out_dir, "r%d" % rank), "w") as f:
        json.dump([ms, total, int(n), [int(w) for w in widths]], f)
    td.barrier()
    td.destroy_process_group()


def test_two_gloo_ranks_take_max_time_and_total_nodes(tmp_path):
    port = _free_port()
    mp.spawn(_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    import json
    r = [json.load(open(tmp_path / ("r%d" % k))) for k in range(2)]
    for ms, total, n, _ in r:
        assert ms == 20.0                       # the slower rank
        assert total == float(r[0][2] + r[1][2])  # all ranks' nodes
    assert r[0][3] != r[1][3]                   # distinct seeded shares
