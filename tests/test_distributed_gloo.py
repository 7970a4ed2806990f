"""The multi-rank path on CPU: two gloo ranks draw disjoint trajectory ranges
(the oracle stands in for each rank's GPU), combine their sub-ensemble sums
with paper_2503_12749_gb300.distributed, and must reproduce the single-process
result on the whole range."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_path):
    import torch.distributed as dist

    import oracle
    import workloads as wl
    from paper_2503_12749_gb300 import distributed as D
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    net = wl.small_network(12, r=0.8, t2=0.9, seed=4)
    per_rank, n_sub, K1 = 1500, 6, 64          # 1500 is not a multiple of n_sub
    e0, E = D.rank_range(rank, world, per_rank, first=11)
    n, nS = oracle.samples(net.T, net.r, net.seed_s, e0, E, 1)
    acc, cnt = oracle.accumulate_gf(n, nS, e0, n_sub, K1, 1)
    acc_all, cnt_all = D.combine_accumulators(acc, cnt)
    if rank == 0:
        np.savez(out_path, acc=acc_all, cnt=cnt_all)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_the_single_run(tmp_path, orc):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    import workloads as wl
    from paper_2503_12749_gb300 import distributed as D
    out = str(tmp_path / "combined.npz")
    mp.spawn(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True)
    got = np.load(out)
    net = wl.small_network(12, r=0.8, t2=0.9, seed=4)
    n, nS = orc.samples(net.T, net.r, net.seed_s, 11, 3000, 1)
    acc, cnt = orc.accumulate_gf(n, nS, 11, 6, 64, 1)
    assert np.array_equal(got["cnt"], cnt)
    # the combined sums differ from the single pass only by summation order
    assert np.allclose(got["acc"], acc, rtol=1e-12, atol=1e-12)
    P1 = orc.invert(got["acc"], got["cnt"])[0]
    P0 = orc.invert(acc, cnt)[0]
    assert np.allclose(P1, P0, rtol=1e-10, atol=1e-13)


def test_rank_ranges_are_disjoint_and_cover():
    from paper_2503_12749_gb300 import distributed as D
    ranges = [D.rank_range(r, 4, 1000, first=5) for r in range(4)]
    assert ranges[0] == (5, 1000)
    ends = [a + b for a, b in ranges]
    assert all(ends[i] == ranges[i + 1][0] for i in range(3))
    with pytest.raises(ValueError):
        D.rank_range(4, 4, 10)
