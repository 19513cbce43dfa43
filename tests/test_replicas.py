"""CPU tests of the replica path (one process per GPU, no data exchange): the
measurement's reduction over world_size-2 gloo ranks, distinct slice batches
per rank, and the reference arm's silent exit on ranks other than 0."""
import os
import socket
import subprocess
import sys

import numpy as np
import torch.multiprocessing as mp

from paper_2603_20611_b300 import replicas, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    seconds = [0.5, 0.75][rank]
    evals = [1.0e9, 3.0e9][rank]
    t, e = replicas.reduce_timing(seconds, evals)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
        f.write(f"{t!r} {e!r}")


def test_reduce_over_two_gloo_ranks(tmp_path):
    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        t, e = (float(x) for x in (tmp_path / f"r{r}.txt").read_text().split())
        assert t == 0.75 and e == 4.0e9  # slowest rank's time, every rank's evaluations
    # whole-job throughput = all ranks' work / slowest rank's time
    assert 4.0e9 / 0.75 > max(1.0e9 / 0.5, 3.0e9 / 0.75)


def test_single_process_reduction_is_identity():
    assert replicas.reduce_timing(0.25, 7.0) == (0.25, 7.0)


def test_ranks_render_distinct_batches():
    seeds = {replicas.batch_seed(r, k) for r in range(8) for k in range(64)}
    assert len(seeds) == 8 * 64
    a = synth.slice_batch(replicas.batch_seed(0, 0), 256, 256, 16)
    b = synth.slice_batch(replicas.batch_seed(1, 0), 256, 256, 16)
    assert len(a) == len(b) == 16 and not np.array_equal(np.sort(a), np.sort(b))


def test_reference_arm_is_silent_on_other_ranks():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2"],
                       env=env, capture_output=True, text=True, timeout=120)
    assert p.returncode == 0 and p.stdout.strip() == ""


def _rank_dies_main(rank, port, out_dir):
    import datetime

    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=2, timeout=datetime.timedelta(seconds=10))
    if rank == 1:
        os._exit(3)  # a rank that fails between steps, before the measurement's reduction
    try:
        replicas.reduce_timing(0.5, 1.0e9)
        outcome = "returned"
    except Exception as e:  # the survivor learns of it from the process group
        outcome = "error " + type(e).__name__
    with open(os.path.join(out_dir, "r0.txt"), "w") as f:
        f.write(outcome)
    os._exit(0)


def test_a_dead_rank_surfaces_as_an_error_not_a_hang(tmp_path):
    """A rank that exits before the reduction makes the other rank's reduction
    raise within the process group's timeout instead of waiting forever."""
    import time
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank_dies_main, args=(r, port, str(tmp_path))) for r in range(2)]
    t0 = time.monotonic()
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(not p.is_alive() for p in procs)
    assert procs[1].exitcode == 3 and procs[0].exitcode == 0
    assert (tmp_path / "r0.txt").read_text().startswith("error")
    assert time.monotonic() - t0 < 120
