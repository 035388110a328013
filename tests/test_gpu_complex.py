"""GPU parity of the complex types (section 2.1: c, z, cz, zc) through the C
ABI: every element bit-identical to the oracle's rounding sequence and within
its error bound of the exact value, for every schedule the planner offers
(warp-mapped tiles, slot-table tiles, index-walk tiles through the
allocation-free entry, multi-row and streaming copies)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1607_01249_gb300 import build as ttc_build
from paper_1607_01249_gb300 import inputs
from paper_1607_01249_gb300 import ttc
from paper_1607_01249_gb300.inputs import Problem
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu

PAIRS = [("c64", "c64"), ("c128", "c128"), ("c64", "c128"), ("c128", "c64")]
SCALARS = [(1.0, 0.0), (1.7 - 0.6j, 0.0), (1.7 - 0.6j, 0.4 + 0.25j), (-0.8, 0.5), (0.3j, -1.1 + 0.7j)]


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    ttc_build.build()
    ttc.lib()


def shapes():
    """Several tiles and a ragged tail on each side; index 0 moved and kept."""
    return [((1, 0), (301, 157)), ((2, 0, 1), (37, 29, 41)), ((0, 2, 1), (45, 33, 27)),
            ((1, 3, 0, 2), (13, 22, 9, 17)), ((3, 1, 0, 2), (7, 31, 5, 19)), ((4, 2, 0, 3, 1), (9, 6, 11, 5, 7)),
            ((0, 1, 3, 2), (3, 1, 70, 40))]


def check(p, seed, plan=None, dist="uniform"):
    A, B0 = H.make_inputs(p, seed, dist)
    got, _ = H.run_gpu(p, A, B0, plan=plan)
    want, _ = H.oracle_mirror(p, A, B0)
    bitcopy = p.alpha == 1.0 and p.beta == 0.0 and p.dtype_in == p.dtype_out
    ok, msg = H.compare_bits(got, want, p.dtype_out, nan_as_nan=not bitcopy)
    assert ok, f"{p}: mirror {msg}"
    ok, msg = H.tolerance_check(p, A, B0, got)
    assert ok, f"{p}: tolerance {msg}"


@pytest.mark.parametrize("din,dout", PAIRS)
@pytest.mark.parametrize("k", range(len(SCALARS)))
def test_complex_pairs_every_shape(din, dout, k):
    alpha, beta = SCALARS[k]
    for i, (perm, sizes) in enumerate(shapes()):
        p = Problem(perm=perm, sizes=sizes, dtype_in=din, dtype_out=dout, alpha=alpha, beta=beta)
        check(p, 100 * k + i)


@pytest.mark.parametrize("din,dout", PAIRS)
def test_complex_every_candidate_schedule(din, dout):
    for i, (perm, sizes) in enumerate(shapes()):
        p = Problem(perm=perm, sizes=sizes, dtype_in=din, dtype_out=dout, alpha=1.7 - 0.6j, beta=0.4 + 0.25j)
        plan = ttc.Plan(p.perm, p.sizes, p.dtype_in, p.dtype_out, p.alpha, p.beta)
        kernels = set()
        for c in range(plan.info()["ncandidates"]):
            plan.select(c)
            kernels.add(plan.info()["kernel"])
            assert plan.verify_schedule() == "", (p, c)
            check(p, 700 + i, plan=plan)
        assert kernels


@pytest.mark.parametrize("din,dout", PAIRS)
def test_complex_outer_sizes_leave_the_rest_of_B(din, dout):
    g = inputs.rng(41)
    for trial in range(4):
        N = int(g.integers(2, 5))
        perm = inputs.random_perm(N, g)
        sizes = tuple(int(g.integers(3, 24)) for _ in range(N))
        oa = tuple(s + int(g.integers(0, 4)) for s in sizes)
        ob = tuple(sizes[q] + int(g.integers(0, 4)) for q in perm)
        p = Problem(perm=perm, sizes=sizes, dtype_in=din, dtype_out=dout, alpha=0.5 + 2j, beta=-0.25j,
                    outer_a=oa, outer_b=ob)
        check(p, 50 + trial)     # the mirror starts from the same B, so bytes outside the sub-tensor must match


@pytest.mark.parametrize("din,dout", PAIRS)
def test_complex_noalloc_entry_runs_the_index_walk(din, dout):
    p = Problem(perm=(2, 0, 1), sizes=(37, 29, 41), dtype_in=din, dtype_out=dout, alpha=1.7 - 0.6j, beta=0.5j)
    plan = ttc.Plan(p.perm, p.sizes, p.dtype_in, p.dtype_out, p.alpha, p.beta)
    A, B0 = H.make_inputs(p, 9)
    dA, dB = H.to_device(A, din), H.to_device(B0, dout)
    plan.execute_noalloc(dA, dB)
    torch.cuda.synchronize()
    want, _ = H.oracle_mirror(p, A, B0)
    ok, msg = H.compare_bits(H.to_host(dB, dout), want, dout, True)
    assert ok, msg


def test_complex_beta_zero_never_reads_B_and_bitcopy_keeps_patterns():
    p = Problem(perm=(1, 2, 0), sizes=(33, 17, 25), dtype_in="c64", dtype_out="c64", alpha=1.5 - 0.5j)
    A, _ = H.make_inputs(p, 3)
    B0 = np.full(p.vol_b, complex(np.nan, np.inf), np.complex64)
    got, _ = H.run_gpu(p, A, B0)
    assert np.all(np.isfinite(got.view(np.float32)))
    # alpha = 1, beta = 0: the bits of every part move unchanged (NaN payloads, -0, subnormals)
    q = Problem(perm=(1, 0), sizes=(70, 90), dtype_in="c128", dtype_out="c128")
    A = H.make_inputs(q, 4)[0]
    parts = A.view(np.uint64)
    parts[:6] = [0x7FF0000000000123, 0xFFF8000000000456, 0x8000000000000000, 1, 0x7FF0000000000000, 3]
    got, _ = H.run_gpu(q, A, np.zeros(q.vol_b, np.complex128))
    want, _ = H.oracle_mirror(q, A, np.zeros(q.vol_b, np.complex128))
    assert got.tobytes() == want.tobytes()


def test_complex_plans_refused_where_unsupported():
    with pytest.raises(ttc.TTCError) as ei:
        ttc.Plan((1, 0), (4, 4), "f32", "f32", 1.0 + 1.0j)
    assert ei.value.name == "TTC_ERR_UNSUPPORTED_DTYPE"
    with pytest.raises(ttc.TTCError) as ei:
        ttc.Plan((1, 0), (4, 4), "c64", "f32")
    assert ei.value.name == "TTC_ERR_UNSUPPORTED_DTYPE"
    plan = ttc.Plan((1, 0), (64, 64), "c64", "c64", 2j)
    A = torch.zeros(64 * 64, dtype=torch.complex64, device="cuda")
    B = torch.zeros(64 * 64, dtype=torch.complex64, device="cuda")
    with pytest.raises(ttc.TTCError) as ei:
        ttc.Batch().add(plan, A, B)
    assert ei.value.name == "TTC_ERR_UNSUPPORTED_DTYPE"


def test_complex_requests_through_the_server():
    """Complex requests never join a batched epoch; they get launches of
    their own beside batched real requests and match the oracle."""
    probs = [Problem(perm=(1, 0), sizes=(40, 30), dtype_in="c64", dtype_out="c64", alpha=1j, beta=0.5),
             Problem(perm=(2, 0, 1), sizes=(9, 8, 7)),
             Problem(perm=(2, 0, 1), sizes=(19, 28, 7), dtype_in="c128", dtype_out="c64", alpha=0.3 - 1j),
             Problem(perm=(1, 0), sizes=(33, 31), dtype_in="bf16", dtype_out="bf16", alpha=2.0)]
    srv = ttc.Server(1 << 30, 2, 4096)
    data = []
    for i, p in enumerate(probs):
        plan = ttc.Plan(p.perm, p.sizes, p.dtype_in, p.dtype_out, p.alpha, p.beta)
        A, B0 = H.make_inputs(p, 60 + i)
        dA, dB = H.to_device(A, p.dtype_in), H.to_device(B0, p.dtype_out)
        data.append((p, A, B0, dB, plan, srv.submit(plan, dA, dB)))
    srv.drain(30_000_000)
    for p, A, B0, dB, plan, t in data:
        assert srv.poll(t, 0)
        want, _ = H.oracle_mirror(p, A, B0)
        ok, msg = H.compare_bits(H.to_host(dB, p.dtype_out), want, p.dtype_out, True)
        assert ok, (p, msg)
    assert srv.stats()["completed"] == len(probs)
    srv.close()


@pytest.mark.parametrize("case", [c for c in inputs.complex_cases() if c.tag in ("C3p1", "C5p0")],
                         ids=lambda c: f"{c.tag}/{c.dtype_in}>{c.dtype_out}/b{int(c.beta != 0)}")
def test_full_size_complex_case_sampled(case):
    """The benchmark's full-size problems, in the configuration the bench
    times (its selected schedule): sampled elements against the oracle's
    definition, computed one by one on the host."""
    plan = ttc.Plan(case.perm, case.sizes, case.dtype_in, case.dtype_out, case.alpha, case.beta)
    A = inputs.tensor_for(case.dtype_in, case.n, 5)
    B0 = inputs.tensor_for(case.dtype_out, case.n, 6)
    dA, dB = H.to_device(A, case.dtype_in), H.to_device(B0, case.dtype_out)
    plan.execute(dA, dB)
    torch.cuda.synchronize()
    got = H.to_host(dB, case.dtype_out)
    g = inputs.rng(77)
    N = len(case.sizes)
    sB = case.sizes_b
    # a sample of B offsets; map each back to its A element through the definition
    offs = g.integers(0, case.n, 4000)
    offs[:2] = [0, case.n - 1]
    strideA = np.cumprod((1,) + case.sizes[:-1])
    strideB = np.cumprod((1,) + sB[:-1])
    j = [(offs // strideB[d]) % sB[d] for d in range(N)]
    i = [None] * N
    for d in range(N):
        i[case.perm[d]] = j[d]
    offA = sum(i[k] * strideA[k] for k in range(N))
    sub = Problem(perm=(0,), sizes=(offs.size,), dtype_in=case.dtype_in, dtype_out=case.dtype_out,
                  alpha=case.alpha, beta=case.beta)
    want, _ = H.oracle_mirror(sub, np.ascontiguousarray(A[offA]), np.ascontiguousarray(B0[offs]))
    ok, msg = H.compare_bits(np.ascontiguousarray(got[offs]), want, case.dtype_out, True)
    assert ok, msg


def crafted_doubles(n, g):
    """binary64 values around every case of the binary64 -> binary32 rounding:
    exponents from the binary32 subnormal range to past its overflow, exact
    ties (even and odd kept parts), carries into the next binade, the largest
    finite binary32 and the halfway point above it, zeros, subnormals,
    infinities and NaN."""
    e = g.integers(860, 1190, n).astype(np.uint64)
    frac = g.integers(0, 1 << 52, n, dtype=np.uint64)
    sign = g.integers(0, 2, n).astype(np.uint64) << np.uint64(63)
    bits = sign | (e << np.uint64(52)) | frac
    k = n // 8
    tie = np.uint64(1 << 28)
    bits[:k] = (bits[:k] & ~np.uint64((1 << 29) - 1)) | tie                     # exact ties
    bits[k:2 * k] |= np.uint64((1 << 29) - 1) << np.uint64(0)                    # round up with carries
    bits[2 * k:2 * k + 8] = np.array([0x47EFFFFFE0000000, 0x47EFFFFFF0000000, 0xC7EFFFFFF0000000,
                                      0x47EFFFFFEFFFFFFF, 0x3810000000000000, 0x380FFFFFF0000000,
                                      0x3800000000000000, 0x36A0000000000000], dtype=np.uint64)
    bits[2 * k + 8:2 * k + 16] = np.array([0, 1 << 63, 1, 0x000FFFFFFFFFFFFF, 0x7FF0000000000000,
                                           0xFFF0000000000000, 0x7FF8000000000001, 0x7FF0000000000001],
                                          dtype=np.uint64)
    return bits.view(np.float64)


def crafted_floats(n, g):
    """binary32 values of every class: normal numbers over the whole exponent
    range, subnormals, zeros, infinities and NaN payloads."""
    bits = g.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32)
    bits[:8] = np.array([0, 0x80000000, 1, 0x007FFFFF, 0x00800000, 0x7F7FFFFF, 0x7F800000, 0xFF800000],
                        dtype=np.uint32)
    bits[8:12] = np.array([0x7FC00001, 0x7F800123, 0xFFC00000, 0x80000001], dtype=np.uint32)
    return bits.view(np.float32)


@pytest.mark.parametrize("din,dout", [("f64", "f32"), ("c128", "c64"), ("f32", "f64"), ("c64", "c128")])
@pytest.mark.parametrize("alpha,beta", [(1.0, 0.0), (1.7, 0.0), (1.0, 0.5), (1.7 - 0.6j, 0.4 + 0.25j)])
def test_mixed_type_conversions_on_crafted_values(din, dout, alpha, beta):
    """The widening and narrowing of the mixed types (the paper's sd, ds, cz,
    zc) on values of every class, bit for bit against the oracle's IEEE
    conversions (NaN results compare as NaN)."""
    if din in ("f32", "f64") and isinstance(alpha, complex):
        pytest.skip("complex scalars need complex tensors")
    g = inputs.rng(91)
    p = Problem(perm=(1, 0), sizes=(96, 80), dtype_in=din, dtype_out=dout, alpha=alpha, beta=beta)
    npart = p.n * (2 if din in H.COMPLEX else 1)
    parts = crafted_doubles(npart, g) if din in ("f64", "c128") else crafted_floats(npart, g)
    A = parts.view(inputs.STORAGE[din])
    nb = p.n * (2 if dout in H.COMPLEX else 1)
    bparts = crafted_doubles(nb, g) if dout in ("f64", "c128") else crafted_floats(nb, g)
    B0 = bparts.view(inputs.STORAGE[dout]).copy()
    got, _ = H.run_gpu(p, A, B0)
    want, _ = H.oracle_mirror(p, A, B0)
    ok, msg = H.compare_bits(got, want, dout, nan_as_nan=True)
    assert ok, msg
