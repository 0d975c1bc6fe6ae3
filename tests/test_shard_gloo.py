"""Two-rank (gloo, CPU) check of the multi-GPU decomposition of the operator.

Each rank owns a contiguous half of the transducer positions.  Forward: the
rank's rows of s equal the same rows of the whole operator.  Adjoint: the
all-reduced sum of the ranks' partial z equals the whole adjoint (Alg. 5 is a
sum over positions).  The operator itself is the FP64 oracle here; the test
covers the partition and the exchange, which run on the host.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_2609_29253_gb300 import shard
        from paper_2609_29253_gb300 import workloads as W

        w = W.small_cylinder(n_vox=6, n_angles=2, n_el=3, L=512)
        taps = oracle.taps_for(w)
        ws, (lo, hi) = shard.shard_workload(w, rank, world)
        s_mine, _ = oracle.forward(ws, taps, w.x.astype(np.float64))
        y = np.random.default_rng(5).standard_normal((w.K, w.L))
        z_mine, _ = oracle.adjoint(ws, taps, y[lo:hi])
        z = torch.from_numpy(z_mine.copy())
        shard.allreduce_adjoint(z)
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), s=s_mine, lo=lo, hi=hi, z=z.numpy())
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_shard_range_partitions():
    from paper_2609_29253_gb300 import shard

    for K in (1, 5, 128, 23040):
        for world in (1, 2, 3, 8):
            r = [shard.shard_range(K, i, world) for i in range(world)]
            assert r[0][0] == 0 and r[-1][1] == K
            assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
            sizes = [hi - lo for lo, hi in r]
            assert max(sizes) - min(sizes) <= 1


def test_angle_batches_disjoint_across_ranks():
    from paper_2609_29253_gb300 import shard

    world, steps = 4, 5
    seen = [shard.angle_batches(180, 4, r, world, steps) for r in range(world)]
    for i in range(steps):
        firsts = [float(seen[r][i][0]) for r in range(world)]
        assert len(set(firsts)) == world


def test_two_rank_forward_rows_and_adjoint_allreduce(tmp_path, oracle_mod):
    import oracle
    from paper_2609_29253_gb300 import workloads as W

    world = 2
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, str(tmp_path))) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0, p.exitcode

    w = W.small_cylinder(n_vox=6, n_angles=2, n_el=3, L=512)
    taps = oracle.taps_for(w)
    s_all, _ = oracle.forward(w, taps, w.x.astype(np.float64))
    y = np.random.default_rng(5).standard_normal((w.K, w.L))
    z_all, _ = oracle.adjoint(w, taps, y)
    parts = [np.load(tmp_path / f"rank{r}.npz") for r in range(world)]
    covered = np.zeros(w.K, dtype=int)
    for p in parts:
        lo, hi = int(p["lo"]), int(p["hi"])
        covered[lo:hi] += 1
        np.testing.assert_allclose(p["s"], s_all[lo:hi], rtol=0, atol=1e-12 * np.abs(s_all).max())
        np.testing.assert_allclose(p["z"], z_all, rtol=0, atol=1e-12 * np.abs(z_all).max())
    assert (covered == 1).all()
