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
    """Rank 0 of the reference arm: the oracle on a pool of host threads (one
    per core), one JSON line with the contract's keys."""
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
    """The all-core pool runs the unchanged oracle on contiguous shares of one
    shared sample: the shares tile the sample, and their results put together
    are the single-call result bit for bit."""
    U, W = bench.oracle_sample(3001)
    pool = bench.OraclePool(U, W, cores=3)
    try:
        assert pool.run(1) > 0
        assert pool.cores == 3
        lens = [sh[0][0].shape[0] for sh in pool.shares]
        assert sum(lens) == 3001 and min(lens) > 0
        parts = [oracle.euler_fused(3, 0, 1.4, Us, Ws) for Us, Ws in pool.shares]
    finally:
        pool.close()
    whole = oracle.euler_fused(3, 0, 1.4, U, W)
    for k in range(45):
        np.testing.assert_array_equal(np.concatenate([p[k] for p in parts]), whole[k])


def test_cpu_baseline_runs_and_sweep():
    """The CPU baseline: five timed runs on one thread and on all cores (best
    >= median), the all-core median as the reported value, and the same
    figures at every size of the sweep."""
    import argparse
    res = bench.cpu_baseline(argparse.Namespace(cpu_sample=4096, cpu_seconds=0.2, cpu_cores=2, cpu_sweep="10,12",
                                                cpu_run_seconds=0.02))
    assert res["kind"] == "oracle" and res["cores"] == 2 and res["runs"] == 5
    assert res["best_value"] >= res["value"] > 0
    assert res["single_thread_best"] >= res["single_thread_value"] > 0
    assert set(res["sweep"]) == {"2^10", "2^12"}
    for v in res["sweep"].values():
        assert v["single_best"] >= v["single_median"] > 0 and v["allcore_best"] >= v["allcore_median"] > 0


def _split_worker(rank, world, port, out_dir, n):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    lo, hi = bench.shard_bounds(n, world, rank)
    # this rank's points of ONE seeded field (the benchmark's seed), as the
    # benchmark's --split mode takes them: a prefix of the stream, sliced
    V = [v[lo:hi] for v in synth.euler3d(hi, seed=1809)]
    W = [w[lo:hi] for w in synth.char_weights(hi, 5, seed=1810)]
    U = oracle.cons_from_prim(3, 1.4, V)
    out = oracle.euler_fused(3, 0, 1.4, U, W)
    parts = [None] * world
    dist.all_gather_object(parts, (lo, hi, np.stack(out)))
    if rank == 0:
        np.save(os.path.join(out_dir, "gathered.npy"), np.concatenate([p[2] for p in parts], axis=1))
        np.save(os.path.join(out_dir, "bounds.npy"), np.array([(p[0], p[1]) for p in parts]))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,n", [(2, 5000), (3, 4099)])
def test_one_field_split_into_contiguous_ranges_gives_the_unsplit_result(tmp_path, world, n):
    """Ranks that split one field into contiguous index ranges (no data
    exchange; the result gathered only to check it) give the unsplit result
    bit for bit; every range starts on a 256-point boundary."""
    mp.start_processes(_split_worker, args=(world, _free_port(), str(tmp_path), n), nprocs=world,
                       start_method="spawn", join=True)
    got = np.load(tmp_path / "gathered.npy")
    bounds = np.load(tmp_path / "bounds.npy")
    assert bounds[0][0] == 0 and bounds[-1][1] == n
    assert all(bounds[r][1] == bounds[r + 1][0] for r in range(world - 1))
    assert all(b[0] % bench.SHARD_ALIGN == 0 for b in bounds)
    U = oracle.cons_from_prim(3, 1.4, synth.euler3d(n, seed=1809))
    W = synth.char_weights(n, 5, seed=1810)
    whole = np.stack(oracle.euler_fused(3, 0, 1.4, U, W))
    np.testing.assert_array_equal(got, whole)


def test_shard_bounds_cover_the_field():
    for n in (0, 1, 255, 256, 1000, 1 << 26):
        for world in (1, 2, 3, 8):
            b = [bench.shard_bounds(n, world, r) for r in range(world)]
            assert b[0][0] == 0 and b[-1][1] == n
            assert all(b[r][1] == b[r + 1][0] for r in range(world - 1))
            assert all(lo <= hi and lo % bench.SHARD_ALIGN == 0 for lo, hi in b)
