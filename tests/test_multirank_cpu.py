"""The N > 1 benchmark path on the CPU with two gloo ranks.

With several GPUs the benchmark runs one independent member per rank
(replicas: the time steps of one member never exchange data with another);
the only collectives are the barrier and the max over the ranks' times.
Here each rank advances its replica with the oracle at T10 (the GPU kernels
need a GPU), through bench.py's own rank helpers."""
import io
import os
import socket
import sys
import contextlib

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _replica(seed):
    from oracle import sdc as osdc
    from oracle.swe import SWE, Params
    from paper_1805_07923_gb300 import inputs
    lvl = osdc.Level(SWE(10, 32, 16, Params()), 3)
    u = inputs.initial_state(10, seed=seed)
    for _ in range(2):
        u = osdc.sdc_step(lvl, u, 600.0, 2)
    return u


def _rank_main(rank, ws, port, out_dir):
    import time
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(ws), RANK=str(rank),
                      LOCAL_RANK=str(rank), MLSDC_BENCH_GLOO="1")
    import torch
    import torch.distributed as dist
    import bench
    ws_, rank_, local_ = bench.dist_init()
    assert (ws_, rank_, local_) == (ws, rank, rank)
    t0 = time.perf_counter()
    u = _replica(bench.replica_seed(rank))
    ms = (time.perf_counter() - t0) * 1e3 + 100.0 * rank   # rank 1 is the slow one
    worst = bench.barrier_max(ms, ws, torch.device("cpu"))
    np.save(os.path.join(out_dir, f"rank{rank}.npy"), u)
    np.save(os.path.join(out_dir, f"time{rank}.npy"), np.array([ms, worst]))
    dist.destroy_process_group()


def test_two_gloo_ranks_run_independent_replicas(tmp_path):
    ws = 2
    mp.start_processes(_rank_main, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, join=True,
                       start_method="spawn")
    sys.path.insert(0, ROOT)
    import bench
    times = [np.load(tmp_path / f"time{r}.npy") for r in range(ws)]
    own = [t[0] for t in times]
    # every rank sees the max over ranks
    for t in times:
        assert t[1] == max(own)
    # the job's value counts the units of all ranks over the slowest rank's time
    assert bench.job_value(ws, 7, max(own)) == pytest.approx(2 * 7 / (max(own) * 1e-3))
    # each rank's member is exactly the member a single process computes from
    # that rank's seed (no data crosses ranks), and the members differ
    states = [np.load(tmp_path / f"rank{r}.npy") for r in range(ws)]
    for r in range(ws):
        assert np.array_equal(states[r], _replica(bench.replica_seed(r)))
    assert not np.allclose(states[0], states[1])


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(type("A", (), {"steps": 3, "gpus": 2})())
    assert buf.getvalue() == ""
