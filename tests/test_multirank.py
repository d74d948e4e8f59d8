"""The multi-rank host logic of bench.py on CPU with two gloo ranks: each rank solves its own
independent market (seed = rank) with no collective on the data path; the only collective is the
max over ranks of the timed region, and the whole-job rate counts every rank's units."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    from paper_2406_10262_gb300 import synth
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = {"n_users": 6, "n_items": 30, "n_slots": 4, "iters": 20}
    r = bench.rank_relevance(w, rank)
    # the rank's own market, solved by the oracle (stands in for the GPU of that rank)
    o = oracle.Oracle(w["n_users"], w["n_items"], w["n_slots"], iters=w["iters"], threads=1)
    o.set_relevance(r.astype(np.float64))
    o.set_exposure(synth.dcg_exposure(w["n_slots"]))
    F, _ = o.step(3)
    ms_local = 10.0 + 5.0 * rank  # a slower second rank
    ms = bench.max_over_ranks(ms_local, dist, "cpu")
    rate = bench.whole_job_rate(1000.0, world, ms)
    np.save(os.path.join(out_dir, f"rank{rank}.npy"),
            np.concatenate([[ms, rate, F[-1]], r.ravel()[:8].astype(np.float64)]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_independent_markets(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank_main, args=(rk, 2, port, str(tmp_path))) for rk in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
        assert p.exitcode == 0
    a, b = (np.load(tmp_path / f"rank{rk}.npy") for rk in range(2))
    assert a[0] == b[0] == 15.0                      # max over ranks
    assert a[1] == b[1] == 2 * 1000.0 / 15e-3        # whole-job units per second
    assert not np.array_equal(a[3:], b[3:])          # different markets (seed = rank)
    assert a[2] != b[2]
    sys.path.insert(0, ROOT)
    import bench
    w = {"n_users": 6, "n_items": 30, "n_slots": 4, "iters": 20}
    np.testing.assert_array_equal(a[3:], bench.rank_relevance(w, 0).ravel()[:8])  # reproducible
