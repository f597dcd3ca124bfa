"""The N > 1 benchmark path on CPU: two ranks over gloo (127.0.0.1).

Each catalogue is independent, so N GPUs run N replicas with no data-path
collective; the host logic is what N > 1 adds: every rank draws its own seeded
catalogue, the job's time is the slowest rank's (all_reduce MAX), and the job's
rate counts the catalogues of all ranks.  Each rank here measures its catalogue
with the FP64 oracle on a 16^3 mesh, as a GPU rank would with the library."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402

WORLD = 2
SCALE = 2e-4  # 2 000 galaxies, 10 000 randoms per rank


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _measure(rank):
    import oracle
    from oracle.binning import BinSpec
    gal, ran, geo = bench.make_workload(rank, "shell512_tsc_il", scale=SCALE)
    res = oracle.fft_multipoles(gal, ran, geo, 16, BinSpec(0.0, 0.002, 6), assign="tsc", interlace=True,
                                ell_max=4, workers=1)
    return np.concatenate([[gal.n, ran.n], res.p0, res.p2, res.p4])


def _rank_main(rank, port, out_dir):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=WORLD)
    try:
        row = _measure(rank)
        # a per-rank "time": the slower rank must set the job's time
        t_job = bench.max_over_ranks(1.5 + rank, "cpu")
        rows = [None] * WORLD
        dist.all_gather_object(rows, row.tolist())
        dist.barrier()
        if rank == 0:
            np.save(os.path.join(out_dir, "rows.npy"), np.array(rows))
            np.save(os.path.join(out_dir, "t_job.npy"), np.array([t_job]))
    finally:
        dist.destroy_process_group()


def test_rank_seeds_distinct():
    seeds = [bench.rank_seeds(r, w) for w in ("shell512_tsc_il", "cone256_tsc_il") for r in range(8)]
    flat = [s for pair in seeds for s in pair]
    assert len(set(flat)) == len(flat)
    assert bench.rank_seeds(0) == (4, 5)     # rank 0 is the single-GPU workload


def test_job_rate_counts_all_ranks():
    assert bench.job_rate(1, 10, 2.0) == 5.0
    assert bench.job_rate(4, 10, 2.0) == 20.0


def test_two_gloo_ranks_run_independent_replicas(tmp_path):
    mp.start_processes(_rank_main, args=(_free_port(), str(tmp_path)), nprocs=WORLD, join=True,
                       start_method="spawn")
    rows = np.load(tmp_path / "rows.npy")
    t_job = float(np.load(tmp_path / "t_job.npy")[0])
    assert t_job == 2.5                       # max over ranks of 1.5 and 2.5
    # each rank measured its own catalogue: the same as a single process gets for that rank
    for r in range(WORLD):
        np.testing.assert_array_equal(rows[r], _measure(r))
    assert not np.array_equal(rows[0][2:], rows[1][2:])
    assert rows[0][0] == rows[1][0] == int(10_000_000 * SCALE)
