"""The N > 1 benchmark path on CPU: two gloo ranks, each evaluating its own
independently seeded field (weak scaling, no data exchange), timing combined
as the maximum over ranks."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
import oracle
from paper_1809_09851_gb300 import synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, local = bench.dist_env()
    assert (w, r, local) == (world, rank, rank)
    seed = bench.shard_seed(1809, r)
    n = 1000
    U = oracle.cons_from_prim(3, 1.4, synth.euler3d(n, seed=seed))
    F = oracle.flux(3, -1, 1.4, U)
    # each rank's elapsed time differs; the job time is the slowest rank's
    t = bench.max_over_ranks(0.5 + rank, w)
    np.save(os.path.join(out_dir, f"rank{rank}.npy"), np.stack([U[0][:8], F[4][:8]]))
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as fh:
        fh.write(f"{t}\n")
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_shard_without_exchange(tmp_path):
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    t = [float(open(tmp_path / f"rank{r}.txt").read()) for r in range(world)]
    assert t == [1.5, 1.5]
    a, b = (np.load(tmp_path / f"rank{r}.npy") for r in range(world))
    assert not np.array_equal(a, b)  # independent fields per rank
    # rank 1's field is exactly what a single process draws with rank 1's seed
    U1 = oracle.cons_from_prim(3, 1.4, synth.euler3d(1000, seed=bench.shard_seed(1809, 1)))
    np.testing.assert_array_equal(b[0], U1[0][:8])


def test_reference_arm_other_ranks_do_no_work(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.main(["--impl", "reference", "--steps", "1", "--warmup", "0"]) is None


def test_reference_arm_json_line(capsys):
    """Rank 0 of the reference arm: the oracle on a pool of host worker
    processes, one JSON line with the contract's keys."""
    import json
    res = bench.main(["--impl", "reference", "--steps", "2", "--warmup", "1", "--ref-sample", "4096"])
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line == res
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["cores"] >= 1 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0


def test_oracle_pool_matches_one_process():
    """The worker pool runs the unchanged oracle on contiguous shares of the sample."""
    pool = bench.OraclePool(3000, cores=2)
    try:
        assert pool.run(1) > 0
    finally:
        pool.close()
    bench._orc_init(3000, 2)
    U, W = bench.oracle_sample(3000)
    whole = oracle.euler_fused(3, 0, 1.4, U, W)
    parts = [oracle.euler_fused(3, 0, 1.4, *bench._ORC["chunks"][i]) for i in range(2)]
    for k in range(45):
        np.testing.assert_array_equal(np.concatenate([parts[0][k], parts[1][k]]), whole[k])


def test_cpu_baseline_runs_and_sweep():
    """The CPU baseline: five timed runs on one thread and on all worker
    processes (best >= median), the all-core median as the reported value, and
    the same figures at every size of the sweep."""
    import argparse
    res = bench.cpu_baseline(argparse.Namespace(cpu_sample=4096, cpu_seconds=0.2, cpu_cores=2, cpu_sweep=(10, 12)))
    assert res["kind"] == "oracle" and res["cores"] == 2 and res["runs"] == 5
    assert res["best_value"] >= res["value"] > 0
    assert res["single_thread_best"] >= res["single_thread_value"] > 0
    assert set(res["sweep"]) == {"2^10", "2^12"}
    for v in res["sweep"].values():
        assert v["single_best"] >= v["single_median"] > 0 and v["allcore_best"] >= v["allcore_median"] > 0
