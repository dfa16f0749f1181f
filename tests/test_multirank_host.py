"""The N > 1 bookkeeping of the benchmark on CPU ranks (gloo, world size 2): one independent system
per rank, whole-job value = particle-steps of all ranks / the slowest rank's time; the reference
arm runs on rank 0 only."""
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


def _rank_main(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    # rank r timed 1.5 + r seconds for 1000 * (r + 1) particle-steps
    t, ps = bench.reduce_over_ranks(dist, torch, 1.5 + rank, 1000 * (rank + 1), "cpu")
    args = bench.parse(["--impl", "reference", "--steps", "1", "--warmup", "0"])
    printed = bench.run_reference(args, rank, world) if rank == 1 else None
    with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
        f.write(f"{t} {ps} {printed}")
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_like_the_benchmark(tmp_path):
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn")
    for r in range(2):
        t, ps, printed = open(tmp_path / f"r{r}.txt").read().split()
        assert float(t) == 2.5                 # slowest rank
        assert float(ps) == 3000.0             # all ranks' particle-steps
        assert printed == "None"
