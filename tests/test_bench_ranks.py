"""bench.py's whole-job reduction over ranks (weak scaling, each rank its own batch), with two gloo ranks on the
CPU: the job's time is the slowest rank's and its units are the sum of every rank's."""
import importlib.util
import json
import os
import socket

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out_dir: str):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
        bench = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(bench)
        ms, units = bench.aggregate_over_ranks(10.0 + 5.0 * rank, 100.0 + rank, world)
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump({"ms": ms, "units": units}, f)
    finally:
        dist.destroy_process_group()


def test_aggregate_over_two_gloo_ranks(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    for r in range(world):
        d = json.load(open(tmp_path / f"rank{r}.json"))
        assert d["ms"] == 15.0 and d["units"] == 201.0


def test_single_rank_passes_through():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    assert bench.aggregate_over_ranks(12.5, 7.0, 1) == (12.5, 7.0)
