"""The multi-GPU form of bench.py is replicas only: every rank runs its own
instances with no collective on the data path, and the job's rate is all ranks'
updates over the slowest rank's time.  Only one GPU is available per run, so this
host-side logic is checked here with two gloo ranks on the CPU."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    import gbs_workloads as w
    wl, meshes = bench.workload_arrays(w.workload("batched_64x_M16_d6"), rank)
    units = int(sum(m.n_gates for m in meshes))
    ms = 100.0 * (rank + 1)          # rank 1 is the slower one
    value = bench.aggregate_value(units, ms, ws, torch.device("cpu"))
    np.save(os.path.join(out_dir, f"r{rank}.npy"),
            np.array([value, units] + list(wl.seeds), dtype=np.float64))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_sharding_and_max_over_ranks(tmp_path):
    ws = 2
    mp.spawn(_rank_main, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, join=True)
    r0 = np.load(tmp_path / "r0.npy")
    r1 = np.load(tmp_path / "r1.npy")
    units = r0[1]
    assert r1[1] == units == 64 * 120
    # both ranks report the same whole-job rate: 2 ranks x units over the slower 200 ms
    assert r0[0] == r1[0] == pytest.approx(ws * units / 0.2)
    seeds0, seeds1 = set(r0[2:].astype(int)), set(r1[2:].astype(int))
    assert seeds0 == set(range(100, 164))
    assert len(seeds1) == 64 and not (seeds0 & seeds1)
