"""Redistributing transpose over several GPUs: Eq. 1 (section 1) on a tensor
sharded across ranks, with the result sharded along a different index.

A is split along one of its indices (`shard_a`) into contiguous blocks, one
per rank; B is wanted split along one of its own indices (`shard_b`, a B
position).  Writing m = perm[shard_b] for the A index that B's sharded index
comes from, rank r holds A_r (A with index shard_a restricted to block r) and
must end with B_q for q = r (B with B index shard_b restricted to block q).

Every element of A_r whose index m lies in block q belongs to B_q, at B
position pos_B(shard_a) inside block r.  So the exchange is one all-to-all:

  1. pack: rank r permutes, for every q, the sub-tensor of A_r with i_m in
     block q into a contiguous piece laid out in B's index order (a permute
     plan with A's outer sizes and an offset along index m; alpha applied);
  2. exchange: the pieces travel with one all_to_all (NCCL on GPUs; the
     pieces are staged in local buffers, no peer or multicast access);
  3. unpack: rank q writes the piece from every r into B_q at offset
     lo_r along B position pos_B(shard_a) (an identity permute plan with B's
     outer sizes; beta applied there, so B is read once).

When m == shard_a the shards already line up: each rank transposes its own
shard, with no exchange.  The local steps run through an executor: by
default this library's permute plans (`ttc.Plan`) on the tensors' device;
tests pass the CPU oracle instead to check the bookkeeping without a GPU.
"""
from __future__ import annotations

from dataclasses import dataclass


def blocks(n: int, world: int) -> list:
    """Contiguous near-equal blocks [lo, hi) of range(n) over `world` ranks
    (the first n % world blocks one longer)."""
    base, extra = divmod(n, world)
    out, lo = [], 0
    for r in range(world):
        hi = lo + base + (1 if r < extra else 0)
        out.append((lo, hi))
        lo = hi
    return out


def _strides(ext):
    st, acc = [], 1
    for e in ext:
        st.append(acc)
        acc *= e
    return st


def _numel(ext):
    n = 1
    for e in ext:
        n *= e
    return n


@dataclass
class Piece:
    """One local permute of the redistribution: `sizes` elements of A (A's
    index order) read from `a_off` inside a tensor of outer sizes `outer_a`,
    written under `perm` to `b_off` inside a tensor of outer sizes `outer_b`
    (B's index order)."""
    perm: tuple
    sizes: tuple
    outer_a: tuple
    a_off: int
    outer_b: tuple
    b_off: int
    alpha: float
    beta: float


class Redistribution:
    """The bookkeeping of one rank's redistributing transpose: what it packs
    for every destination, the all-to-all split sizes, and where each
    received piece lands in its B shard."""

    def __init__(self, perm, sizes, shard_a: int, shard_b: int, rank: int, world: int, alpha=1.0, beta=0.0):
        n = len(sizes)
        if sorted(perm) != list(range(n)):
            raise ValueError("perm is not a permutation")
        if not (0 <= shard_a < n and 0 <= shard_b < n):
            raise ValueError("shard index out of range")
        if not (0 <= rank < world):
            raise ValueError("rank out of range")
        self.perm, self.sizes = tuple(perm), tuple(int(s) for s in sizes)
        self.shard_a, self.shard_b, self.rank, self.world = shard_a, shard_b, rank, world
        self.alpha, self.beta = float(alpha), float(beta)
        self.m = self.perm[shard_b]                      # A index behind B's sharded index
        self.pos_a = self.perm.index(shard_a)            # B position of A's sharded index
        self.blk_a = blocks(self.sizes[shard_a], world)
        self.blk_b = blocks(self.sizes[self.m], world)
        lo, hi = self.blk_a[rank]
        self.a_local = tuple(hi - lo if k == shard_a else s for k, s in enumerate(self.sizes))
        qlo, qhi = self.blk_b[rank]
        sB = [self.sizes[p] for p in self.perm]
        self.b_local = tuple(qhi - qlo if d == shard_b else s for d, s in enumerate(sB))
        self.exchange = self.m != shard_a

    # -- no exchange: the shards line up
    def local_piece(self) -> Piece:
        return Piece(self.perm, self.a_local, self.a_local, 0, self.b_local, 0, self.alpha, self.beta)

    # -- pack: the piece of A_r bound for rank q, into the send buffer
    def send_pieces(self):
        st_a = _strides(self.a_local)
        out, off = [], 0
        for q in range(self.world):
            lo, hi = self.blk_b[q]
            sz = tuple(hi - lo if k == self.m else s for k, s in enumerate(self.a_local))
            out_b = tuple(sz[p] for p in self.perm)       # contiguous, B order
            out.append(Piece(self.perm, sz, self.a_local, lo * st_a[self.m], out_b, off, self.alpha, 0.0))
            off += _numel(sz)
        return out

    def send_counts(self):
        return [_numel(p.sizes) for p in self.send_pieces()]

    # -- unpack: the piece from rank r, from the receive buffer into B_q
    def recv_pieces(self):
        st_b = _strides(self.b_local)
        out, off = [], 0
        for r in range(self.world):
            lo, hi = self.blk_a[r]
            sz = tuple(hi - lo if d == self.pos_a else s for d, s in enumerate(self.b_local))
            ident = tuple(range(len(sz)))
            out.append(Piece(ident, sz, sz, off, self.b_local, lo * st_b[self.pos_a], 1.0, self.beta))
            off += _numel(sz)
        return out

    def recv_counts(self):
        return [_numel(p.sizes) for p in self.recv_pieces()]


def ttc_executor(dtype: str):
    """The default executor: this library's permute plans on the tensors'
    device (plans are cached per piece shape)."""
    from . import ttc
    cache = {}
    elsize = {"f32": 4, "f64": 8, "bf16": 2, "c64": 8, "c128": 16}[dtype]

    def run(p: Piece, src, dst, stream=None):
        key = (p.perm, p.sizes, p.outer_a, p.outer_b, p.alpha, p.beta)
        plan = cache.get(key)
        if plan is None:
            plan = ttc.Plan(p.perm, p.sizes, dtype, dtype, p.alpha, p.beta, p.outer_a, p.outer_b)
            cache[key] = plan
        plan.execute(src.data_ptr() + p.a_off * elsize, dst.data_ptr() + p.b_off * elsize, stream)
    return run


def redistributing_transpose(A_local, B_local, perm, sizes, shard_a: int, shard_b: int, alpha=1.0, beta=0.0,
                             group=None, executor=None, dtype: str = "f32"):
    """B_local <- alpha * (this rank's block of B) + beta * B_local, where
    A_local is this rank's block of A along index shard_a and B_local its
    block of B along B position shard_b (flat column-major tensors, torch).
    Collective over `group` (every rank calls it with its own shards)."""
    import torch
    import torch.distributed as tdist
    world = tdist.get_world_size(group)
    rank = tdist.get_rank(group)
    rd = Redistribution(perm, sizes, shard_a, shard_b, rank, world, alpha, beta)
    run = executor or ttc_executor(dtype)
    if not rd.exchange:
        run(rd.local_piece(), A_local, B_local)
        return B_local
    send = torch.empty(sum(rd.send_counts()), dtype=A_local.dtype, device=A_local.device)
    recv = torch.empty(sum(rd.recv_counts()), dtype=A_local.dtype, device=A_local.device)
    for p in rd.send_pieces():
        run(p, A_local, send)
    if send.is_cuda:
        torch.cuda.current_stream().synchronize()
    tdist.all_to_all_single(recv, send, output_split_sizes=rd.recv_counts(), input_split_sizes=rd.send_counts(),
                            group=group)
    for p in rd.recv_pieces():
        run(p, recv, B_local)
    return B_local
