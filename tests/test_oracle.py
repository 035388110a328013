"""Pins of the CPU oracle against things other than itself (no GPU needed).

* numpy.transpose on (slices of) row-major views: the library special case
  that fixes the permutation convention, the column-major layout and the
  meaning of outer sizes (section 1 Eq. 1, fn. 2; section 2.1 Table 1, Fig. 2);
* the 2D textbook transpose, identity, inverse and composition of perms;
* the paper's printed examples (tests/golden/paper_examples.txt);
* exact rational arithmetic (fractions.Fraction) for alpha*a + beta*b;
* torch's own bfloat16 / float8_e4m3fn conversions for the number formats;
* closed forms for the FP8 scale.
"""
import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1607_01249_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- helpers

def rowmajor_view(buf, outer, sizes):
    """Column-major tensor of `sizes` inside an outer tensor `outer`, as the
    equivalent row-major numpy view (axes reversed)."""
    full = buf.reshape(tuple(reversed(outer)))
    return full[tuple(slice(0, s) for s in reversed(sizes))]


def numpy_reference(perm, sizes, A, B, outerA=None, outerB=None):
    """B <- A under perm using np.transpose: B axis a takes A axis q[a] with
    q[a] = N-1-perm[N-1-a] (row-major axes are column-major indices reversed)."""
    N = len(sizes)
    oA = outerA or sizes
    sB = tuple(sizes[p] for p in perm)
    oB = outerB or sB
    q = [N - 1 - perm[N - 1 - a] for a in range(N)]
    Bv = rowmajor_view(B, oB, sB)
    Bv[...] = np.transpose(rowmajor_view(A, oA, sizes), axes=q)
    return B


def rand_outer(sizes, g):
    return tuple(int(s + g.integers(0, 3)) for s in sizes)


def rn_f32_exact(q: Fraction) -> float:
    """Round a rational to the nearest binary32 (ties to even), exactly."""
    if q == 0:
        return 0.0
    s = -1.0 if q < 0 else 1.0
    a = abs(q)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    while Fraction(2) ** e > a:
        e -= 1
    while Fraction(2) ** (e + 1) <= a:
        e += 1
    e = max(e, -126)
    quantum = Fraction(2) ** (e - 23)
    m = a / quantum
    mi = m.numerator // m.denominator
    rem = m - mi
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and mi % 2 == 1):
        mi += 1
    v = mi * quantum
    if v >= Fraction(2) ** 128:
        return s * math.inf
    return s * float(v)


# ------------------------------------------------- permutation semantics

@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_all_perms_vs_numpy_with_outer_sizes(N):
    g = inputs.rng(100 + N)
    for perm in itertools.permutations(range(N)):
        for trial in range(3):
            sizes = tuple(int(x) for x in g.choice([1, 2, 3, 5], size=N))
            oA = rand_outer(sizes, g) if trial else None
            sB = tuple(sizes[p] for p in perm)
            oB = rand_outer(sB, g) if trial == 2 else None
            for dt in (oracle.F32, oracle.F64, oracle.BF16):
                npdt = oracle.NP_DTYPE[dt]
                volA = int(np.prod(oA or sizes))
                volB = int(np.prod(oB or sB))
                A = g.integers(0, 60000, size=volA).astype(npdt)
                canary = g.integers(0, 60000, size=volB).astype(npdt)
                B = canary.copy()
                oracle.permute(perm, sizes, A, B, dtA=dt, dtB=dt, outerA=oA, outerB=oB)
                R = numpy_reference(perm, sizes, A, canary.copy(), oA, oB)
                assert np.array_equal(B.view(np.uint8), R.view(np.uint8)), (perm, sizes, oA, oB)


def test_textbook_2d():
    g = inputs.rng(7)
    s0, s1 = 13, 7
    A = g.standard_normal(s0 * s1).astype(np.float32)
    B = np.zeros(s0 * s1, np.float32)
    oracle.permute((1, 0), (s0, s1), A, B)
    for i in range(s0):
        for j in range(s1):
            assert B[j + i * s1] == A[i + j * s0]


def test_identity_is_copy():
    g = inputs.rng(8)
    for N in range(1, 6):
        sizes = tuple(int(x) for x in g.integers(1, 6, size=N))
        A = g.standard_normal(int(np.prod(sizes))).astype(np.float64)
        B = np.zeros_like(A)
        oracle.permute(tuple(range(N)), sizes, A, B, dtA=oracle.F64, dtB=oracle.F64)
        assert A.tobytes() == B.tobytes()


def test_inverse_and_composition():
    g = inputs.rng(9)
    for N in (3, 4, 5):
        for _ in range(6):
            p1 = inputs.random_perm(N, g)
            p2 = inputs.random_perm(N, g)
            sizes = tuple(int(x) for x in g.integers(1, 6, size=N))
            A = g.standard_normal(int(np.prod(sizes))).astype(np.float32)
            B1 = np.zeros_like(A)
            oracle.permute(p1, sizes, A, B1)
            inv = [0] * N
            for d in range(N):
                inv[p1[d]] = d
            s1 = tuple(sizes[p] for p in p1)
            back = np.zeros_like(A)
            oracle.permute(tuple(inv), s1, B1, back)
            assert back.tobytes() == A.tobytes()
            # p2 applied to B1 equals one transpose of A with c[e] = p1[p2[e]]
            B2 = np.zeros_like(A)
            oracle.permute(p2, s1, B1, B2)
            c = tuple(p1[p2[e]] for e in range(N))
            Bc = np.zeros_like(A)
            oracle.permute(c, sizes, A, Bc)
            assert B2.tobytes() == Bc.tobytes()


def test_paper_printed_examples():
    with open(os.path.join(GOLDEN, "paper_examples.txt")) as f:
        rows = [l for l in f.read().splitlines() if l.strip() and not l.startswith("#")]
    assert len(rows) == 2
    for row in rows:
        name, perm, sizes, lda, ldb, out, cite = [x.strip() for x in row.split("|")]
        perm = tuple(int(x) for x in perm.split(","))
        sizes = tuple(int(x) for x in sizes.split(","))
        lda = None if lda == "-" else tuple(int(x) for x in lda.split(","))
        assert ldb == "-"
        names = out[2:-1].split(",")                 # "B(i2,i1,i0)" -> ["i2","i1","i0"]
        src = [int(nm[1:]) for nm in names]          # B index d holds A index src[d]
        assert tuple(src) == perm, name
        oA = lda or sizes
        sB = [sizes[k] for k in src]
        volA = int(np.prod(oA))
        A = np.arange(volA, dtype=np.float64)        # each element = its own A offset
        B = np.full(int(np.prod(sB)), -1.0)
        oracle.permute(perm, sizes, A, B, dtA=oracle.F64, dtB=oracle.F64, outerA=lda)
        for i in itertools.product(*[range(s) for s in sizes]):
            offA = sum(i[k] * int(np.prod(oA[:k])) for k in range(len(sizes)))
            j = [i[k] for k in src]
            offB = sum(j[d] * int(np.prod(sB[:d])) for d in range(len(sizes)))
            assert B[offB] == offA


# ------------------------------------------------------------ arithmetic

def test_bitcopy_preserves_special_bit_patterns():
    pats = np.array([0x80000000, 0x00000001, 0x807FFFFF, 0x7FC00123, 0xFFA00001, 0x7F800000,
                     0xFF800000, 0x3F800000, 0x00800000, 0x7F7FFFFF], dtype=np.uint32)
    A = np.tile(pats, 3).view(np.float32)
    sizes = (5, 6)
    B = np.zeros(30, np.float32)
    oracle.permute((1, 0), sizes, A, B)
    assert sorted(B.view(np.uint32).tolist()) == sorted(A.view(np.uint32).tolist())


def test_beta0_does_not_read_B():
    g = inputs.rng(11)
    A = g.uniform(-1, 1, 60).astype(np.float32)
    for dt, npdt in ((oracle.F32, np.float32), (oracle.F64, np.float64)):
        Aa = A.astype(npdt)
        B = np.full(60, np.nan, npdt)
        oracle.permute((2, 0, 1), (3, 4, 5), Aa, B, alpha=1.7, beta=0.0, dtA=dt, dtB=dt)
        assert np.all(np.isfinite(B))
        R, S = oracle.permute_exact((2, 0, 1), (3, 4, 5), Aa, np.full(60, np.nan, npdt),
                                    alpha=1.7, beta=0.0, dtA=dt, dtB=dt)
        assert np.all(np.isfinite(R))


def _axpby_case(dt, seed, n=96):
    g = inputs.rng(seed)
    npdt = np.float32 if dt == oracle.F32 else np.float64
    A = g.uniform(-1, 1, n).astype(npdt)
    B0 = g.uniform(-1, 1, n).astype(npdt)
    A[:4] = [0.5, -0.25, 3.0, 1e-3]
    return A, B0


def test_f32_exact_value_matches_rational_arithmetic():
    alpha, beta = 1.7, 0.4
    af, bf = float(np.float32(alpha)), float(np.float32(beta))
    perm, sizes = (1, 2, 0), (4, 6, 4)
    A, B0 = _axpby_case(oracle.F32, 12)
    R, S = oracle.permute_exact(perm, sizes, A, B0.copy(), alpha, beta)
    Bm = B0.copy()
    oracle.permute(perm, sizes, A, Bm, alpha, beta)
    # element-by-element: find each A element's destination from a numpy transpose
    idx = np.arange(A.size, dtype=np.float64)
    dest = numpy_reference(perm, sizes, idx, np.zeros(A.size))       # dest[offB] = offA
    for offB in range(A.size):
        offA = int(dest[offB])
        exact = Fraction(af) * Fraction(float(A[offA])) + Fraction(bf) * Fraction(float(B0[offB]))
        assert R[offB] == float(exact)                                 # correctly rounded
        p = rn_f32_exact(Fraction(af) * Fraction(float(A[offA])))
        mirror = rn_f32_exact(Fraction(bf) * Fraction(float(B0[offB])) + Fraction(p))
        assert float(Bm[offB]) == mirror
        # the reading's primary tolerance: within 2 FP32 ulps of the exact value
        ulp = 2.0 ** (math.floor(math.log2(S[offB])) - 23)
        assert abs(float(Bm[offB]) - R[offB]) <= 2 * ulp


def test_f64_exact_value_matches_rational_arithmetic():
    alpha, beta = 1.7, 0.4
    perm, sizes = (2, 0, 1), (4, 4, 6)
    A, B0 = _axpby_case(oracle.F64, 13)
    R, S = oracle.permute_exact(perm, sizes, A, B0.copy(), alpha, beta, oracle.F64, oracle.F64)
    Bm = B0.copy()
    oracle.permute(perm, sizes, A, Bm, alpha, beta, oracle.F64, oracle.F64)
    idx = np.arange(A.size, dtype=np.float64)
    dest = numpy_reference(perm, sizes, idx, np.zeros(A.size))
    n_exact = 0
    for offB in range(A.size):
        offA = int(dest[offB])
        exact = Fraction(alpha) * Fraction(float(A[offA])) + Fraction(beta) * Fraction(float(B0[offB]))
        ex = float(exact)
        assert abs(R[offB] - ex) <= math.ulp(ex)
        n_exact += R[offB] == ex
        mirror = float(Fraction(beta) * Fraction(float(B0[offB])) + Fraction(alpha * float(A[offA])))
        assert float(Bm[offB]) == mirror
        assert abs(float(Bm[offB]) - R[offB]) <= 1e-15 * S[offB]
    assert n_exact >= 0.95 * A.size


def test_fmaf_is_correctly_rounded():
    g = inputs.rng(14)
    a = g.uniform(-2, 2, 400).astype(np.float32)
    b = g.uniform(-2, 2, 400).astype(np.float32)
    c = (-(a.astype(np.float64) * b)).astype(np.float32)      # heavy cancellation
    c[::2] = g.uniform(-2, 2, 200).astype(np.float32)
    y = oracle.fmaf(a, b, c)
    for k in range(400):
        ex = Fraction(float(a[k])) * Fraction(float(b[k])) + Fraction(float(c[k]))
        assert float(y[k]) == rn_f32_exact(ex)


def test_mixed_f32_to_f64_and_back():
    g = inputs.rng(15)
    A = g.uniform(-1, 1, 60).astype(np.float32)
    B = np.zeros(60, np.float64)
    oracle.permute((1, 0), (6, 10), A, B, dtA=oracle.F32, dtB=oracle.F64)
    assert np.array_equal(B, numpy_reference((1, 0), (6, 10), A.astype(np.float64), np.zeros(60)))
    A64 = g.uniform(-1, 1, 60)
    B32 = np.zeros(60, np.float32)
    oracle.permute((1, 0), (6, 10), A64, B32, alpha=1.7, dtA=oracle.F64, dtB=oracle.F32)
    ref = numpy_reference((1, 0), (6, 10), (1.7 * A64).astype(np.float32), np.zeros(60, np.float32))
    assert np.array_equal(B32, ref)           # numpy's float64->float32 cast is RN


# -------------------------------------------------------- number formats

def test_bf16_encoder_against_torch():
    torch = pytest.importorskip("torch")
    hi = np.arange(1 << 16, dtype=np.uint32) << 16
    lows = np.array([0, 1, 0x7FFF, 0x8000, 0x8001, 0xFFFF], dtype=np.uint32)
    pats = (hi[:, None] | lows[None, :]).ravel()
    pats = np.concatenate([pats, inputs.rng(16).integers(0, 1 << 32, size=1 << 20,
                                                         dtype=np.uint64).astype(np.uint32)])
    x = pats.view(np.float32)
    ours = oracle.bf16_from_f32(x)
    theirs = torch.from_numpy(x.copy()).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    nan = np.isnan(x)
    assert np.array_equal(ours[~nan], theirs[~nan])
    ours_f = (ours.astype(np.uint32) << 16).view(np.float32)
    assert np.all(np.isnan(ours_f[nan]))


def test_e4m3_decode_all_codes_against_torch():
    torch = pytest.importorskip("torch")
    codes = np.arange(256, dtype=np.uint8)
    ours = oracle.e4m3_to_f32(codes)
    theirs = torch.from_numpy(codes.copy()).view(torch.float8_e4m3fn).float().numpy()
    both_nan = np.isnan(ours) & np.isnan(theirs)
    assert np.array_equal(np.isnan(ours), np.isnan(theirs))
    assert np.array_equal(ours[~both_nan], theirs[~both_nan])
    assert ours[0x7E] == 448.0 and ours[0x01] == 2.0 ** -9 and ours[0x08] == 2.0 ** -6
    assert np.sum(np.isnan(ours)) == 2


def test_e4m3_encoder_against_torch_and_saturation():
    torch = pytest.importorskip("torch")
    g = inputs.rng(17)
    vals = oracle.e4m3_to_f32(np.arange(0, 0x7F, dtype=np.uint8)).astype(np.float64)
    mids = (vals[:-1] + vals[1:]) / 2                  # exact ties (representable in f32)
    mids32 = mids.astype(np.float32)
    near = np.concatenate([np.nextafter(mids32, np.float32(0)), np.nextafter(mids32, np.float32(1e9))])
    mag = np.exp(g.uniform(np.log(2.0 ** -12), np.log(464.0), size=1 << 20)).astype(np.float32)
    x = np.concatenate([vals.astype(np.float32), mids32, near, mag, [0.0, 2.0 ** -11, 464.0]]).astype(np.float32)
    x = np.concatenate([x, -x]).astype(np.float32)
    ours = oracle.e4m3_from_f32(x)
    theirs = torch.from_numpy(x.copy()).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    assert np.array_equal(ours, theirs)
    # satfinite (OCP definition): everything beyond the largest finite value -> +-448
    big = np.array([464.0001, 479.9, 480.0, 1e6, 3.4e38, np.inf], np.float32)
    assert np.all(oracle.e4m3_from_f32(big) == 0x7E)
    assert np.all(oracle.e4m3_from_f32(-big) == 0xFE)
    assert oracle.e4m3_from_f32(np.array([np.nan], np.float32))[0] & 0x7F == 0x7F


def test_fp8_scale_closed_forms():
    g = inputs.rng(18)
    A = g.uniform(-1, 1, 240).astype(np.float32)
    A[17] = -448.0 * 2.0 ** -5                        # amax = 14 -> scale 2^-5 exactly
    scale, amax = oracle.fp8_scale((4, 6, 10), A)
    assert amax == 14.0 and scale == 2.0 ** -5
    B = np.zeros(240, np.uint8)
    oracle.permute((2, 0, 1), (4, 6, 10), A, B, dtA=oracle.F32, dtB=oracle.E4M3, fp8_scale=scale)
    ref = numpy_reference((2, 0, 1), (4, 6, 10), oracle.e4m3_from_f32(A * np.float32(32.0)),
                          np.zeros(240, np.uint8))
    assert np.array_equal(B, ref)
    assert 0xFE in B                                  # the amax element codes to -448
    # dequantised error bound: |q*scale - a| <= 2^-4 |a| + scale * 2^-10
    deq = oracle.e4m3_to_f32(B).astype(np.float64) * scale
    exact = numpy_reference((2, 0, 1), (4, 6, 10), A.astype(np.float64), np.zeros(240))
    assert np.all(np.abs(deq - exact) <= 2.0 ** -4 * np.abs(exact) + scale * 2.0 ** -10)
    # alpha enters the amax
    s2, a2 = oracle.fp8_scale((4, 6, 10), A, alpha=2.0)
    assert a2 == 28.0 and s2 == 2.0 ** -4
    # degenerate amax -> scale 1; NaN ignored
    assert oracle.fp8_scale((8,), np.zeros(8, np.float32)) == (1.0, 0.0)
    Z = np.ones(8, np.float32); Z[3] = np.inf
    assert oracle.fp8_scale((8,), Z)[0] == 1.0
    Z = np.ones(8, np.float32) * 0.5; Z[3] = np.nan; Z[5] = 224.0
    assert oracle.fp8_scale((8,), Z) == (0.5, 224.0)
    # an outer-size sub-tensor only looks at its own elements
    big = np.zeros(6 * 6, np.float32); big[5] = 1000.0; big[7] = 7.0
    assert oracle.fp8_scale((3, 3), big, outerA=(6, 6))[1] == 7.0


def test_bf16_output_rounding_of_axpby():
    g = inputs.rng(19)
    A = g.uniform(-1, 1, 120).astype(np.float32)
    B0 = oracle.bf16_from_f32(g.uniform(-1, 1, 120).astype(np.float32))
    B = B0.copy()
    oracle.permute((1, 0), (10, 12), A, B, 1.7, 0.4, oracle.F32, oracle.BF16)
    dest = numpy_reference((1, 0), (10, 12), np.arange(120.0), np.zeros(120))
    af, bf = np.float32(1.7), np.float32(0.4)
    for offB in range(120):
        a = A[int(dest[offB])]
        b = (np.uint32(B0[offB]) << np.uint32(16)).view(np.float32)
        p = rn_f32_exact(Fraction(float(af)) * Fraction(float(a)))
        r = rn_f32_exact(Fraction(float(bf)) * Fraction(float(b)) + Fraction(p))
        assert B[offB] == oracle.bf16_from_f32(np.array([r], np.float32))[0]


def test_rejects_invalid_problems():
    A = np.zeros(8, np.float32)
    B = np.zeros(8, np.float32)
    with pytest.raises(ValueError):
        oracle.permute((0, 0), (2, 4), A, B)
    with pytest.raises(ValueError):
        oracle.permute((1, 0), (2, 4), A, B, outerA=(1, 4))
    with pytest.raises(ValueError):
        oracle.permute((1, 0), (2, 4), A, np.zeros(8, np.uint8), beta=0.5, dtB=oracle.E4M3)
