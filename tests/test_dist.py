"""The redistributing transpose over several ranks (paper_1607_01249_gb300/dist.py)
on the CPU: Eq. 1 on a tensor sharded along one A index, the result sharded
along a B index.  The local permutes run through the oracle (an executor the
module takes), so these tests check the partition, the all-to-all split sizes
and where every piece lands, against the oracle's transpose of the whole
tensor sliced to each rank's block.  First with the exchange simulated in one
process for 2, 3 and 4 ranks; then with two gloo ranks and a real
all_to_all."""
import itertools
import os
import socket
import sys

import numpy as np
import pytest

import oracle
from paper_1607_01249_gb300 import dist

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def oracle_executor():
    def run(p, src, dst, stream=None):
        a = src.numpy() if hasattr(src, "numpy") else src
        b = dst.numpy() if hasattr(dst, "numpy") else dst
        oracle.permute(p.perm, p.sizes, a[p.a_off:], b[p.b_off:], p.alpha, p.beta, oracle.F64, oracle.F64,
                       p.outer_a, p.outer_b)
    return run


def colmajor(flat, sizes):
    return flat.reshape(tuple(reversed(sizes)))      # row-major view, indices reversed


def shard(x, sizes, k, lo, hi):
    """Block [lo, hi) of index k of the column-major tensor x, as a flat
    contiguous column-major tensor."""
    v = colmajor(x, sizes)
    ax = len(sizes) - 1 - k
    sl = [slice(None)] * len(sizes)
    sl[ax] = slice(lo, hi)
    return np.ascontiguousarray(v[tuple(sl)]).ravel()


def whole_result(perm, sizes, A, B0, alpha, beta):
    sB = [sizes[p] for p in perm]
    B = B0.copy()
    oracle.permute(perm, sizes, A, B, alpha, beta, oracle.F64, oracle.F64)
    return B, sB


def simulate(perm, sizes, shard_a, shard_b, world, alpha, beta, seed):
    """Every rank's pack, the all-to-all as list slicing, every rank's
    unpack; returns each rank's B block and the expected one."""
    rng = np.random.default_rng(seed)
    n = int(np.prod(sizes))
    A = rng.uniform(-1, 1, n)
    sB = [sizes[p] for p in perm]
    B0 = rng.uniform(-1, 1, n)
    want, _ = whole_result(perm, sizes, A, B0, alpha, beta)
    run = oracle_executor()
    rds = [dist.Redistribution(perm, sizes, shard_a, shard_b, r, world, alpha, beta) for r in range(world)]
    a_blocks = [shard(A, sizes, shard_a, *rds[0].blk_a[r]) for r in range(world)]
    b_blocks = [shard(B0, sB, shard_b, *rds[0].blk_b[q]) for q in range(world)]
    wants = [shard(want, sB, shard_b, *rds[0].blk_b[q]) for q in range(world)]
    if not rds[0].exchange:
        for r in range(world):
            run(rds[r].local_piece(), a_blocks[r], b_blocks[r])
        return b_blocks, wants
    sends = []
    for r in range(world):
        buf = np.zeros(sum(rds[r].send_counts()))
        for p in rds[r].send_pieces():
            run(p, a_blocks[r], buf)
        sends.append(buf)
    for q in range(world):
        # the all-to-all: rank q receives the q-th part of every rank's send buffer
        parts = []
        for r in range(world):
            cnt = rds[r].send_counts()
            at = sum(cnt[:q])
            parts.append(sends[r][at:at + cnt[q]])
        assert [len(x) for x in parts] == rds[q].recv_counts()
        recv = np.concatenate(parts) if parts else np.zeros(0)
        for p in rds[q].recv_pieces():
            run(p, recv, b_blocks[q])
    return b_blocks, wants


CASES = [
    ((1, 0), (37, 23)),
    ((2, 0, 1), (7, 11, 13)),
    ((0, 2, 1), (5, 9, 8)),
    ((3, 1, 0, 2), (4, 6, 5, 7)),
    ((1, 3, 0, 2), (6, 5, 3, 4)),
]


@pytest.mark.parametrize("world", [2, 3, 4])
@pytest.mark.parametrize("perm,sizes", CASES)
def test_simulated_exchange_matches_the_oracle(perm, sizes, world):
    n = len(sizes)
    for shard_a, shard_b in itertools.product(range(n), range(n)):
        got, want = simulate(perm, sizes, shard_a, shard_b, world, 1.7, 0.4, seed=shard_a * 7 + shard_b)
        for q in range(world):
            assert np.array_equal(got[q], want[q]), (perm, sizes, shard_a, shard_b, world, q)


def test_blocks_cover_the_index_and_allow_empty_ones():
    assert dist.blocks(10, 3) == [(0, 4), (4, 7), (7, 10)]
    assert dist.blocks(2, 4) == [(0, 1), (1, 2), (2, 2), (2, 2)]
    got, want = simulate((1, 0), (3, 2), 0, 0, 4, 1.0, 0.0, seed=1)
    for q in range(4):
        assert np.array_equal(got[q], want[q])


def test_counts_are_symmetric_across_ranks():
    perm, sizes, world = (2, 0, 1), (7, 11, 13), 3
    rds = [dist.Redistribution(perm, sizes, 2, 1, r, world) for r in range(world)]
    for r in range(world):
        for q in range(world):
            assert rds[r].send_counts()[q] == rds[q].recv_counts()[r]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    import torch
    import torch.distributed as tdist
    sys.path.insert(0, ROOT)
    from paper_1607_01249_gb300 import dist as D
    from tests import test_dist as T
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bad = []
        for ci, (perm, sizes) in enumerate(T.CASES):
            n = len(sizes)
            for shard_a, shard_b in itertools.product(range(n), range(n)):
                rng = np.random.default_rng(100 + ci)
                A = rng.uniform(-1, 1, int(np.prod(sizes)))
                B0 = rng.uniform(-1, 1, A.size)
                want, sB = T.whole_result(perm, sizes, A, B0, -0.5, 0.25)
                rd = D.Redistribution(perm, sizes, shard_a, shard_b, rank, world)
                a_loc = torch.from_numpy(T.shard(A, sizes, shard_a, *rd.blk_a[rank]))
                b_loc = torch.from_numpy(T.shard(B0, sB, shard_b, *rd.blk_b[rank]))
                D.redistributing_transpose(a_loc, b_loc, perm, sizes, shard_a, shard_b, -0.5, 0.25,
                                           executor=T.oracle_executor(), dtype="f64")
                if not np.array_equal(b_loc.numpy(), T.shard(want, sB, shard_b, *rd.blk_b[rank])):
                    bad.append(f"{perm} {sizes} {shard_a} {shard_b}")
        with open(os.path.join(out_dir, f"r{rank}"), "w") as f:
            f.write("\n".join(bad) if bad else "ok")
        tdist.barrier()
    finally:
        tdist.destroy_process_group()


def test_two_gloo_ranks_exchange_with_all_to_all(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    world = 2
    mp.start_processes(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    for r in range(world):
        assert (tmp_path / f"r{r}").read_text() == "ok"
