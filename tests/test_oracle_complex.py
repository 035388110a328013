"""Pins of the oracle's complex path (section 2.1: single-complex "c",
double-complex "z", mixed "cz" / "zc") against things other than itself:

* numpy.transpose of complex arrays (layout and permutation of the pairs) and
  numpy's own complex64 <-> complex128 casts (the mixed types);
* closed forms: multiplying by i, -i or 2i and updating with beta = i are
  exact, so their results are fixed bit for bit;
* the real oracle (pinned in test_oracle.py): with real scalars a complex
  tensor is a real tensor with an extra leading index of extent 2;
* exact rational arithmetic (fractions.Fraction) for the definition of the
  complex product and for the fixed rounding sequence;
* numpy's complex128 arithmetic for alpha*a + beta*b.
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1607_01249_gb300 import inputs
from tests.test_oracle import numpy_reference, rand_outer, rn_f32_exact

CDT = {"c64": (oracle.C64, np.complex64, oracle.F32, np.float32),
       "c128": (oracle.C128, np.complex128, oracle.F64, np.float64)}


def crand(n, g, npdt):
    parts = g.uniform(-1, 1, 2 * n)
    return parts.astype(np.float32 if npdt == np.complex64 else np.float64).view(npdt)


def vol(sizes, outer=None):
    return int(np.prod(outer or sizes, dtype=np.int64))


def same_bits(x, y):
    return x.dtype == y.dtype and x.shape == y.shape and x.tobytes() == y.tobytes()


# ------------------------------------------------ layout and permutation

@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_complex_bitcopy_vs_numpy_with_outer_sizes(dt, N):
    odt, npdt, _, _ = CDT[dt]
    g = inputs.rng(200 + N)
    for perm in itertools.permutations(range(N)):
        sizes = tuple(int(x) for x in g.choice([1, 2, 3, 5], size=N))
        oA = rand_outer(sizes, g)
        sB = tuple(sizes[p] for p in perm)
        oB = rand_outer(sB, g)
        A = crand(vol(sizes, oA), g, npdt)
        canary = crand(vol(sB, oB), g, npdt)
        got = oracle.permute_complex(perm, sizes, A, canary.copy(), 1.0, 0.0, odt, odt, oA, oB)
        want = numpy_reference(perm, sizes, A, canary.copy(), oA, oB)
        assert same_bits(got, want), (perm, sizes)


@pytest.mark.parametrize("din,dout", [("c64", "c128"), ("c128", "c64")])
def test_mixed_complex_types_match_numpy_casts(din, dout):
    """cz widens each part exactly; zc rounds each part once to nearest (numpy
    casts complex128 -> complex64 part by part with IEEE rounding)."""
    g = inputs.rng(210)
    perm, sizes = (2, 0, 1), (3, 4, 5)
    A = crand(vol(sizes), g, CDT[din][1])
    B = np.zeros(vol(sizes), CDT[dout][1])
    got = oracle.permute_complex(perm, sizes, A, B, 1.0, 0.0, CDT[din][0], CDT[dout][0])
    want = numpy_reference(perm, sizes, A.astype(CDT[dout][1]), np.zeros_like(B))
    assert same_bits(got, want)


# ---------------------------------------------------------- closed forms

@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_multiplying_by_i_is_exact(dt):
    """(x + iy) * i = -y + ix, (x + iy) * (-i) = y - ix, (x + iy) * 2i =
    -2y + 2ix: every rounding in the sequence is exact, so these fix the signs
    and the operand order of the cross terms."""
    odt, npdt, _, _ = CDT[dt]
    g = inputs.rng(220)
    perm, sizes = (1, 2, 0), (4, 3, 5)
    A = crand(vol(sizes), g, npdt)
    T = numpy_reference(perm, sizes, A, np.zeros_like(A))
    for alpha, want in ((1j, -T.imag + 1j * T.real), (-1j, T.imag - 1j * T.real),
                        (2j, -2 * T.imag + 2j * T.real)):
        got = oracle.permute_complex(perm, sizes, A, np.zeros_like(A), alpha, 0.0, odt, odt)
        assert same_bits(got, want.astype(npdt)), alpha


@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_beta_update_closed_forms(dt):
    """alpha = 0: beta = i turns b into i*b, beta = -1 into -b, beta = 1 - i
    into (u + v) + i(v - u) up to one rounding per part."""
    odt, npdt, _, _ = CDT[dt]
    g = inputs.rng(230)
    perm, sizes = (1, 0), (6, 7)
    A = crand(vol(sizes), g, npdt)
    B0 = crand(vol(sizes), g, npdt)
    got = oracle.permute_complex(perm, sizes, A, B0.copy(), 0.0, 1j, odt, odt)
    assert same_bits(got, (-B0.imag + 1j * B0.real).astype(npdt))
    got = oracle.permute_complex(perm, sizes, A, B0.copy(), 0.0, -1.0, odt, odt)
    assert same_bits(got, (-B0).astype(npdt))
    got = oracle.permute_complex(perm, sizes, A, B0.copy(), 0.0, 1 - 1j, odt, odt)
    want = (B0.real + B0.imag) + 1j * (B0.imag - B0.real)     # numpy: one rounding per part
    assert same_bits(got, want.astype(npdt))


@pytest.mark.parametrize("din,dout", [("c64", "c64"), ("c128", "c128"), ("c64", "c128"), ("c128", "c64")])
def test_real_scalars_reduce_to_the_real_oracle(din, dout):
    """With real alpha and beta a complex tensor of sizes s is a real tensor of
    sizes (2,) + s whose new leading index stays in place."""
    g = inputs.rng(240)
    perm, sizes = (2, 0, 3, 1), (3, 4, 2, 5)
    oA = rand_outer(sizes, g)
    sB = tuple(sizes[p] for p in perm)
    oB = rand_outer(sB, g)
    A = crand(vol(sizes, oA), g, CDT[din][1])
    B0 = crand(vol(sB, oB), g, CDT[dout][1])
    for alpha, beta in ((1.7, 0.0), (1.7, 0.4), (-0.3, 2.5)):
        got = oracle.permute_complex(perm, sizes, A, B0.copy(), alpha, beta, CDT[din][0], CDT[dout][0], oA, oB)
        Br = B0.copy().view(CDT[dout][3])
        oracle.permute((0,) + tuple(p + 1 for p in perm), (2,) + sizes, A.view(CDT[din][3]), Br, alpha, beta,
                       CDT[din][2], CDT[dout][2], (2,) + oA, (2,) + oB)
        assert same_bits(got, Br.view(CDT[dout][1])), (alpha, beta)


def test_beta0_does_not_read_B_and_rejects_real_types():
    perm, sizes = (1, 0), (5, 3)
    g = inputs.rng(250)
    A = crand(15, g, np.complex64)
    B = np.full(15, complex(np.nan, np.nan), np.complex64)
    got = oracle.permute_complex(perm, sizes, A, B, 1.5 - 0.5j, 0.0, oracle.C64, oracle.C64)
    assert np.all(np.isfinite(got.view(np.float32)))
    with pytest.raises(ValueError):
        oracle.permute_complex(perm, sizes, A, B, 1.0, 0.0, oracle.C64, oracle.F32)


# ------------------------------------------------------- exact arithmetic

def _cases(dt, seed):
    odt, npdt, _, _ = CDT[dt]
    g = inputs.rng(seed)
    perm, sizes = (2, 0, 1), (3, 4, 5)
    A = crand(vol(sizes), g, npdt)
    B0 = crand(vol(sizes), g, npdt)
    A[:3] = [0.5 - 0.25j, 3.0 + 1e-3j, -0.0 + 0.0j]
    idx = np.arange(A.size, dtype=np.float64)
    dest = numpy_reference(perm, sizes, idx, np.zeros(A.size))       # dest[offB] = offA
    return odt, npdt, perm, sizes, A, B0, dest


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("alpha,beta", [(1.7 - 0.6j, 0.0), (1.7 - 0.6j, 0.4 + 0.25j), (0.3j, -1.1 + 0.0j),
                                        (2.0, 0.5j)])
def test_complex_exact_value_is_the_definition(dt, alpha, beta):
    """The exact oracle against the definition of the complex product in exact
    rational arithmetic, (ar + i ai)(x + i y) = (ar x - ai y) + i(ar y + ai x),
    with the scalars rounded part by part to the compute type."""
    odt, npdt, perm, sizes, A, B0, dest = _cases(dt, 260)
    rnd = (lambda v: float(np.float32(v))) if dt == "c64" else float
    ar, ai, br, bi = (Fraction(rnd(v)) for v in (alpha.real if isinstance(alpha, complex) else alpha,
                                                  complex(alpha).imag, complex(beta).real, complex(beta).imag))
    R, S = oracle.permute_complex_exact(perm, sizes, A, B0.copy(), alpha, beta, odt, odt)
    bnz = complex(beta) != 0
    for offB in range(A.size):
        a = A[int(dest[offB])]
        x, y = Fraction(float(a.real)), Fraction(float(a.imag))
        u, v = (Fraction(float(B0[offB].real)), Fraction(float(B0[offB].imag))) if bnz else (0, 0)
        re = ar * x - ai * y + br * u - bi * v
        im = ar * y + ai * x + br * v + bi * u
        for got, ex in ((R[offB].real, re), (R[offB].imag, im)):
            e = float(ex)
            assert abs(got - e) <= math.ulp(e) if e != 0 else abs(got) <= 2.0 ** -1000
        sre = abs(ar * x) + abs(ai * y) + abs(br * u) + abs(bi * v)
        assert S[offB, 0] == pytest.approx(float(sre), rel=1e-15)


def _seq(ops, rn):
    """The fixed rounding sequence of the complex update, each step evaluated
    exactly and then rounded by `rn`."""
    ar, ai, br, bi, x, y, u, v, bnz = ops
    re, im = rn(ar * x), rn(ar * y)
    if ai != 0:
        re, im = rn(-ai * y + Fraction(re)), rn(ai * x + Fraction(im))
    if bnz:
        re, im = rn(br * u + Fraction(re)), rn(br * v + Fraction(im))
        if bi != 0:
            re, im = rn(-bi * v + Fraction(re)), rn(bi * u + Fraction(im))
    return re, im


@pytest.mark.parametrize("din,dout", [("c64", "c64"), ("c128", "c128"), ("c64", "c128"), ("c128", "c64")])
@pytest.mark.parametrize("alpha,beta", [(1.7 - 0.6j, 0.0), (1.7 - 0.6j, 0.4 + 0.25j), (-0.9, 0.7 - 1.3j)])
def test_complex_rounding_sequence_in_rational_arithmetic(din, dout, alpha, beta):
    """Every step of the oracle's sequence is an exactly rounded operation:
    re-evaluated with Fractions and an explicit round-to-nearest-even it gives
    the same bits, and the result lies within the sequence's error bound of the
    exact value (4 roundings in the compute type plus one to B's type)."""
    odt, npdt, perm, sizes, A, _, dest = _cases(din, 270)
    g = inputs.rng(271)
    B0 = crand(A.size, g, CDT[dout][1])
    wide = "c128" in (din, dout)
    rn = float if wide else rn_f32_exact
    cast = (lambda v: float(v)) if wide else (lambda v: float(np.float32(v)))
    a_, b_ = complex(alpha), complex(beta)
    ar, ai, br, bi = (Fraction(cast(v)) for v in (a_.real, a_.imag, b_.real, b_.imag))
    got = oracle.permute_complex(perm, sizes, A, B0.copy(), alpha, beta, odt, CDT[dout][0])
    R, S = oracle.permute_complex_exact(perm, sizes, A, B0.copy(), alpha, beta, odt, CDT[dout][0])
    eps_c = 2.0 ** -53 if wide else 2.0 ** -24
    eps_o = 2.0 ** -24 if dout == "c64" else 2.0 ** -53
    for offB in range(A.size):
        a = A[int(dest[offB])]
        ops = (ar, ai, br, bi, Fraction(float(a.real)), Fraction(float(a.imag)),
               Fraction(float(B0[offB].real)), Fraction(float(B0[offB].imag)), b_ != 0)
        re, im = _seq(ops, rn)
        if dout == "c64" and wide:
            re, im = float(np.float32(re)), float(np.float32(im))      # one more rounding, double -> float
        assert float(got[offB].real) == re and float(got[offB].imag) == im, offB
        for k, part in enumerate((got[offB].real, got[offB].imag)):
            ex = R[offB].real if k == 0 else R[offB].imag
            assert abs(float(part) - ex) <= 4 * eps_c * S[offB, k] + eps_o * abs(ex) + 1e-300


@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_complex_exact_value_against_numpy_complex_arithmetic(dt):
    """numpy's complex128 alpha*a + beta*b (textbook product, rounded steps)
    agrees with the exact oracle within a few double ulps of the scale."""
    odt, npdt, perm, sizes, A, B0, _ = _cases(dt, 280)
    alpha, beta = 1.7 - 0.6j, 0.4 + 0.25j
    if dt == "c64":
        alpha = complex(np.complex64(alpha))
        beta = complex(np.complex64(beta))
    R, S = oracle.permute_complex_exact(perm, sizes, A, B0.copy(), alpha, beta, odt, odt)
    TA = numpy_reference(perm, sizes, A.astype(np.complex128), np.zeros(A.size, np.complex128))
    want = alpha * TA + beta * B0.astype(np.complex128)
    assert np.all(np.abs(want.real - R.real) <= 8 * 2.0 ** -53 * S[:, 0])
    assert np.all(np.abs(want.imag - R.imag) <= 8 * 2.0 ** -53 * S[:, 1])
