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


def _rank_systems(rank, world, port, out_dir):
    # each rank steps its own seeded system (the benchmark's workload shape at a small size, on the
    # CPU oracle) and the whole-job figure adds up both ranks' particle-steps
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import hashlib
    import time

    import bench
    import oracle as O

    args = bench.parse(["--n-each", "300", "--steps", "2", "--warmup", "0"])
    system = bench.workload(args, seed=1 + rank)
    st = O.init_state(system)
    ps = 0
    t0 = time.perf_counter()
    for _ in range(2):
        ps += st.n
        st, _ = O.step(system, st)
    el = time.perf_counter() - t0
    t, total = bench.reduce_over_ranks(dist, torch, el, ps, "cpu")
    digest = hashlib.sha256(st.x.tobytes() + st.ids.tobytes()).hexdigest()
    with open(os.path.join(out_dir, f"s{rank}.txt"), "w") as f:
        f.write(f"{system.seed} {ps} {total} {t >= el} {digest}")
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_step_independent_seeded_systems(tmp_path):
    port = _free_port()
    mp.start_processes(_rank_systems, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn")
    rows = [open(tmp_path / f"s{r}.txt").read().split() for r in range(2)]
    assert [int(r[0]) for r in rows] == [1, 2]                 # one seed per rank
    assert rows[0][4] != rows[1][4]                            # different trajectories
    ps = [int(r[1]) for r in rows]
    assert all(float(r[2]) == float(sum(ps)) for r in rows)    # the job's particle-steps on every rank
    assert all(r[3] == "True" for r in rows)                   # the job time is the slowest rank's
