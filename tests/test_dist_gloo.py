"""Multi-rank path on the CPU: world_size 2 over gloo.

Each rank transports its own history-id range (the oracle stands in for the
per-GPU engine here) and the tallies are summed with the same helper bench.py
uses; the result must equal one process running all histories, bit for bit.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2605_25963_gb300 import dist as D
from paper_2605_25963_gb300 import workloads as W

N_PER_RANK = 6000


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    from oracle import oracle as O
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        m = O.Mesh.build(O.Det(**W.BARE_CYLINDER.as_dict()))
        t = O.Tables.build(W.MATERIAL_CODES)
        src = O.Source(kind=W.SRC_POINT, pos=W.BARE_POINT_100.pos)
        r = O.transport(m, t, src, 662.0, N_PER_RANK, history_offset=D.history_offset(rank, N_PER_RANK),
                        n_threads=2)
        counts = {k: r.tally[k] for k in ("n_hist", "n_fep", "n_zero", "n_over", "n_err", "n_segments",
                                          "n_interactions")}
        out, spec, fepe, sigma = D.reduce_tallies(counts, r.spectrum)
        q.put((rank, out, spec.tolist(), fepe, sigma))
    finally:
        dist.destroy_process_group()


def test_two_rank_partition_equals_single_run(orc):
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=240) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    m = orc.Mesh.build(orc.Det(**W.BARE_CYLINDER.as_dict()))
    t = orc.Tables.build(W.MATERIAL_CODES)
    ref = orc.transport(m, t, orc.Source(kind=W.SRC_POINT, pos=W.BARE_POINT_100.pos), 662.0, world * N_PER_RANK)
    for rank, out, spec, fepe, sigma in res:
        for k, v in out.items():
            assert v == ref.tally[k], (rank, k)
        assert np.array_equal(np.array(spec), ref.spectrum)
        assert fepe == ref.fepe and sigma == pytest.approx(ref.sigma, rel=1e-12, abs=0)


def test_split_range_covers_everything():
    for n in (0, 1, 7, 1000, 10 ** 9 + 3):
        for w in (1, 2, 3, 8):
            parts = [D.split_range(n, w, r) for r in range(w)]
            assert parts[0][0] == 0
            for (a, ca), (b, _) in zip(parts[:-1], parts[1:]):
                assert a + ca == b
            assert sum(c for _, c in parts) == n
    assert D.history_offset(3, 100, base=7) == 307
