"""Pins of the contraction oracle (the definition TTGT computes, section 1)
against things other than itself: brute-force loops over every index value
on small integer-valued tensors (sums exact in float64), matrix product,
outer product and dot product in closed form, and the beta update."""
import itertools

import numpy as np
import pytest

import oracle
from paper_1607_01249_gb300 import inputs


def brute(modes_a, A, sa, modes_b, B, sb, modes_c, sc, alpha, beta, C):
    ext = dict(zip(modes_a, sa))
    ext.update(zip(modes_b, sb))
    ext.update(zip(modes_c, sc))
    summed = [m for m in ext if m not in modes_c]
    out = np.zeros(int(np.prod(sc, dtype=np.int64)))

    def off(modes, sizes, val):
        o, st = 0, 1
        for m, s in zip(modes, sizes):
            o += val[m] * st
            st *= s
        return o

    for cv in itertools.product(*[range(ext[m]) for m in modes_c]):
        val = dict(zip(modes_c, cv))
        acc = 0.0
        for kv in itertools.product(*[range(ext[m]) for m in summed]):
            val.update(zip(summed, kv))
            acc += A[off(modes_a, sa, val)] * B[off(modes_b, sb, val)]
        o = off(modes_c, sc, dict(zip(modes_c, cv)))
        out[o] = alpha * acc + (beta * C[o] if beta else 0.0)
    return out


CASES = [
    ((0, 1), (1, 2), (0, 2)),                   # matrix product
    ((1, 0), (2, 1), (2, 0)),                   # transposed operands and result
    ((0, 3, 1, 4), (4, 2, 3), (2, 0, 1)),       # two contracted labels, permuted
    ((0, 1), (2, 3), (3, 0, 2, 1)),             # outer product (nothing contracted)
    ((0, 1, 2), (2, 0, 1), ()),                 # full contraction to a scalar
    ((5, 1, 0), (1, 3), (3, 0, 5)),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_contraction_oracle_matches_brute_force(case):
    ma, mb, mc = CASES[case]
    g = inputs.rng(300 + case)
    ext = {m: int(g.integers(1, 5)) for m in set(ma) | set(mb) | set(mc)}
    sa, sb, sc = (tuple(ext[m] for m in ms) for ms in (ma, mb, mc))
    A = g.integers(-4, 5, int(np.prod(sa, dtype=np.int64))).astype(np.float64)
    B = g.integers(-4, 5, int(np.prod(sb, dtype=np.int64))).astype(np.float64)
    C = g.integers(-4, 5, int(np.prod(sc, dtype=np.int64))).astype(np.float64)
    for alpha, beta in ((1.0, 0.0), (2.0, -3.0)):
        got = oracle.contract(ma, A, sa, mb, B, sb, mc, C, sc, alpha, beta)
        want = brute(ma, A, sa, mb, B, sb, mc, sc, alpha, beta, C)
        assert np.array_equal(got, want), (case, alpha, beta)       # integer data: every sum is exact


def test_contraction_oracle_closed_forms():
    g = inputs.rng(310)
    A = g.standard_normal(6 * 7)
    B = g.standard_normal(7 * 5)
    # C = A B (column-major 6x7 times 7x5)
    got = oracle.contract((0, 1), A, (6, 7), (1, 2), B, (7, 5), (0, 2), None, (6, 5))
    want = (A.reshape(6, 7, order="F") @ B.reshape(7, 5, order="F")).reshape(-1, order="F")
    assert np.allclose(got, want, rtol=1e-14, atol=1e-14)
    # outer product: C[i, j] = a[i] b[j]
    a, b = g.standard_normal(9), g.standard_normal(4)
    got = oracle.contract((0,), a, (9,), (1,), b, (4,), (0, 1), None, (9, 4))
    assert np.array_equal(got, np.outer(a, b).reshape(-1, order="F"))
    # dot product
    got = oracle.contract((0,), a, (9,), (0,), a, (9,), (), None, ())
    assert np.isclose(got[0], float(np.dot(a, a)), rtol=1e-15)
    # the absolute contraction bounds the plain one
    r = oracle.contract((0, 1), A, (6, 7), (1, 2), B, (7, 5), (0, 2), None, (6, 5))
    s = oracle.contract((0, 1), A, (6, 7), (1, 2), B, (7, 5), (0, 2), None, (6, 5), absolute=True)
    assert np.all(np.abs(r) <= s + 1e-12)
