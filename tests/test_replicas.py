"""Multi-process host logic of a replicated run, on CPU with gloo (world size 2).

A multi-GPU run is N independent replicas (no exchange step on the path):
each rank renders its own seeded copy of a workload of the same size, the
per-rank times are reduced by their maximum, and the whole-job rate is the
frames of all ranks over the slowest rank's time. These tests run that logic
as two gloo processes; no GPU is touched.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    from paper_2508_18540_gb300 import replicas as R
    from paper_2508_18540_gb300 import synth as S

    r, w, local = R.env_rank()
    assert (r, w, local) == (rank, world, rank)
    dist.init_process_group("gloo", init_method="env://", rank=r, world_size=w)
    try:
        # each rank's own scene: same sizes, different seed
        wl = S.workload_display(seed=R.replica_seed(2, r), n=3000, res=32, N=4, V=3)
        shapes = (wl.scene.n, wl.N, wl.camera.Nx, wl.camera.Ny, wl.views.Vx)
        checksum = float(np.asarray(wl.scene.means, dtype=np.float64).sum())
        got = [None] * w
        dist.all_gather_object(got, (shapes, checksum))

        R.barrier(w)
        # a slower rank 1: the job runs at its pace
        per_rank_ms = 4.0 + 3.0 * r
        mx = R.max_over_ranks(per_rank_ms, w)
        rate = R.job_rate(mx, w)
        np.save(os.path.join(out_dir, "rank%d.npy" % r),
                np.array([mx, rate, got[0][1], got[1][1]] + list(got[0][0]) + list(got[1][0]), dtype=np.float64))
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas(tmp_path):
    import torch.multiprocessing as mp

    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    rows = [np.load(tmp_path / ("rank%d.npy" % r)) for r in range(world)]
    for row in rows:
        mx, rate = row[0], row[1]
        assert mx == 7.0                                   # max over ranks, seen by both
        assert rate == pytest.approx(1000.0 / 7.0 * 2)     # frames of both ranks / slowest time
        assert row[2] != row[3]                            # the replicas render different scenes
        assert np.array_equal(row[4:9], row[9:14])         # of the same sizes
    assert np.array_equal(rows[0], rows[1])


def test_single_process_helpers(monkeypatch):
    from paper_2508_18540_gb300 import replicas as R

    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert R.env_rank() == (0, 1, 0)
    assert R.max_over_ranks(3.5, 1) == 3.5
    assert R.job_rate(2.0, 1) == 500.0
    assert R.job_rate(2.0, 4, units_per_step=45) == pytest.approx(90000.0)
    assert R.replica_seed(2, 0) == 2 and R.replica_seed(2, 3) == 5
    for bad in (0.0, -1.0, float("nan")):
        with pytest.raises(ValueError):
            R.job_rate(bad, 1)
    with pytest.raises(ValueError):
        R.job_rate(1.0, 0)
    with pytest.raises(ValueError):
        R.replica_seed(2, -1)


def test_reference_arm_other_ranks_do_no_work(monkeypatch):
    """Under a multi-process launch the reference arm runs on rank 0 only;
    the other ranks return without work."""
    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    assert bench.run_reference(None) is None
