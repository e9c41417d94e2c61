"""The N > 1 path of the bench on CPU: two ranks over gloo (127.0.0.1) run the replica
aggregation (max of the step times, sum of the units) and the reference arm's rank rule,
as `torchrun --nproc-per-node 2 bench.py` would on GPUs."""
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


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 10.0 + 2.0 * rank                  # rank 1 is the slower replica
    units = 1.0e9 * (1 + rank)              # replicas may process different unit counts
    out[rank] = bench.replica_rate(ms, units, world, dist)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replica_rate():
    world, port = 2, _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        ms, rate = res[rank]
        assert ms == 12.0                    # max over ranks
        assert rate == pytest.approx(3.0e9 / 12e-3)   # all units / max time


def test_single_rank_replica_rate():
    import bench
    ms, rate = bench.replica_rate(8.0, 4.0e9, 1)
    assert ms == 8.0 and rate == pytest.approx(4.0e9 / 8e-3)


def test_reference_arm_other_ranks_exit_quietly(capsys, monkeypatch):
    """Under torchrun only rank 0 runs the reference arm; the others return at once."""
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setattr("sys.argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    bench.run_reference(bench.parse())
    assert capsys.readouterr().out == ""
