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


def test_reference_arm_json_line(capsys, monkeypatch):
    """Rank 0 of the reference arm times the oracle on a bounded sample and prints one
    JSON line with the contract's keys (here on a 48^3 twin for speed)."""
    import json
    import bench
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setattr("sys.argv", ["bench.py", "--impl", "reference", "--n", "48", "--nt", "6",
                                     "--steps", "1", "--warmup", "0"])
    bench.run_reference(bench.parse())
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"]
    assert line["metric"] == "Gpts/s fwd+adjoint" and line["unit"] == "Gpts/s"
    assert line["config"]["workload"].startswith("salt_3d")
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
