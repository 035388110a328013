"""GPU parity of the tensor-core GEMM that consumes the packing routine
(ttc_packed_gemm_*): the panel P must be exactly the oracle's FP32 -> BF16
permutation (round to nearest even) of A's sub-tensor, and C = alpha * P * Bm
within the FP32-accumulation bound gamma_(K+1) * |alpha| |P| |Bm| (taken with
a unit roundoff of 2^-23, one bit more than round-to-nearest, since the
tensor cores' internal accumulation order and rounding are not specified)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1607_01249_gb300 import build as ttc_build
from paper_1607_01249_gb300 import inputs
from paper_1607_01249_gb300 import ttc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    ttc_build.build()
    ttc.lib()


def bf16_to_f64(bits):
    return (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def run(perm, sizes, rank_m, n, alpha=1.0, outer=None, seed=0, classic=False):
    g = inputs.rng(seed)
    oa = outer or sizes
    A = g.uniform(-1, 1, int(np.prod(oa, dtype=np.int64))).astype(np.float32)
    gemm = ttc.PackedGemm(perm, sizes, rank_m, n, alpha, outer)
    gemm.classic(classic)
    inf = gemm.info()
    M, K = inf["m"], inf["k"]
    Bm = oracle.bf16_from_f32(g.uniform(-1, 1, K * n).astype(np.float32))
    dA = torch.from_numpy(A).cuda()
    dB = torch.from_numpy(Bm.view(np.int16)).cuda()
    dC = torch.full((M * n,), float("nan"), device="cuda")
    gemm.execute(dA, dB, dC)
    torch.cuda.synchronize()
    gemm.check()
    got = dC.cpu().numpy().astype(np.float64).reshape(n, M).T          # column-major M x N
    # P: the oracle's permutation with the BF16 downcast, as an M x K column-major matrix
    sB = [sizes[p] for p in perm]
    P = np.zeros(int(np.prod(sB, dtype=np.int64)), np.uint16)
    oracle.permute(perm, sizes, A, P, 1.0, 0.0, oracle.F32, oracle.BF16, outer, None)
    Pm = bf16_to_f64(P).reshape(K, M).T
    Bmm = bf16_to_f64(Bm).reshape(n, K).T
    want = alpha * (Pm @ Bmm)
    scale = abs(alpha) * (np.abs(Pm) @ np.abs(Bmm))
    u = 2.0 ** -23
    gamma = (K + 1) * u / (1 - (K + 1) * u)
    err = np.abs(got - want)
    bad = ~(err <= gamma * scale + 1e-30)
    assert not bad.any(), (perm, sizes, rank_m, n, int(bad.sum()), float(np.nanmax(err)))
    return gemm


# both kernels: the default (the warp-specialised one -- Bm by TMA, the
# pack by its own warps -- where the pack loads 16 bytes at a time) and the
# register-staged one
KERNELS = [False, True]


@pytest.mark.parametrize("classic", KERNELS)
def test_packed_gemm_plain_matrix_one_tile(classic):
    run((0, 1), (128, 64), 1, 128, seed=1, classic=classic)


@pytest.mark.parametrize("classic", KERNELS)
def test_packed_gemm_ragged_edges_and_transposed_operand(classic):
    # A stored K x M: the panel is its transpose; M, N and K all ragged
    run((1, 0), (72, 200), 1, 150, alpha=1.5, seed=2, classic=classic)


@pytest.mark.parametrize("classic", KERNELS)
def test_packed_gemm_permuted_4d_operand(classic):
    # A[a, e, b, f] contracted over (e, f): M = a * b, K = e * f (the TTGT layout)
    run((0, 2, 1, 3), (20, 8, 13, 9), 2, 96, alpha=-0.75, seed=3, classic=classic)


@pytest.mark.parametrize("classic", KERNELS)
def test_packed_gemm_sub_block_with_outer_sizes(classic):
    # a 300 x 136 block of a larger 320 x 160 matrix (the packing of section 2.1, Fig. 2)
    run((0, 1), (300, 136), 1, 257, outer=(320, 160), seed=4, classic=classic)


@pytest.mark.parametrize("classic", KERNELS)
def test_packed_gemm_several_k_stages_and_tiles(classic):
    run((1, 0, 2), (16, 40, 24), 2, 300, seed=5, classic=classic)          # M = 640, K = 24
    run((2, 0, 1), (32, 24, 16), 1, 200, seed=6, classic=classic)          # M = 16, K = 768 (12 stages)
    run((1, 0), (520, 1000), 1, 700, seed=7, classic=classic)              # many tiles per CTA, ragged


@pytest.mark.parametrize("case", inputs.packed_gemm_cases(), ids=lambda c: c["tag"])
def test_packed_gemm_at_bench_size_sampled(case):
    """The bench's packed GEMMs at full size (a 4096 x 2048 block of an
    8192^2 matrix times 2048 x 4096, its transposed storage, the 48^4 TTGT
    operand): 96 sampled entries of C against the definition on the
    operands rounded to BF16, and the default kernel (the warp-specialised
    one where the pack loads 16 bytes at a time) equal bit for bit to the
    register-staged one."""
    perm, sizes, outer, rank_m, n = case["perm"], case["sizes"], case["outer"], case["rank_m"], case["n"]
    g = inputs.rng(41)
    oa = outer or sizes
    A = g.uniform(-1, 1, int(np.prod(oa, dtype=np.int64))).astype(np.float32)
    outs = []
    for classic in (False, True):
        gemm = ttc.PackedGemm(perm, sizes, rank_m, n, 1.0, outer).classic(classic)
        inf = gemm.info()
        M, K = inf["m"], inf["k"]
        if not outs:
            Bm = oracle.bf16_from_f32(g.uniform(-1, 1, K * n).astype(np.float32))
            dA = torch.from_numpy(A).cuda()
            dB = torch.from_numpy(Bm.view(np.int16)).cuda()
        dC = torch.full((M * n,), float("nan"), device="cuda")
        gemm.execute(dA, dB, dC)
        torch.cuda.synchronize()
        gemm.check()
        outs.append(dC.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])
    got = outs[0].astype(np.float64).reshape(n, M).T
    # P[m, k]: the A element the packing maps to (row m, column k), rounded to BF16
    sB = [sizes[p] for p in perm]
    stA = np.cumprod((1,) + tuple(oa[:-1]))
    Ar = bf16_to_f64(oracle.bf16_from_f32(A))
    Bmm = bf16_to_f64(Bm).reshape(n, K).T
    nm = rank_m

    def a_offset(m, k):
        # B order index (m's digits over the first rank_m B indices, k's over the rest) -> A offset
        idx, off = [0] * len(sizes), 0
        for d in range(nm):
            idx[perm[d]] = m % sB[d]
            m //= sB[d]
        for d in range(nm, len(perm)):
            idx[perm[d]] = k % sB[d]
            k //= sB[d]
        return int(sum(i * s for i, s in zip(idx, stA)))

    u = 2.0 ** -23
    gamma = (K + 1) * u / (1 - (K + 1) * u)
    for _ in range(96):
        m, j = int(g.integers(0, M)), int(g.integers(0, n))
        row = np.array([Ar[a_offset(m, k)] for k in range(K)])
        want = float(row @ Bmm[:, j])
        scale = float(np.abs(row) @ np.abs(Bmm[:, j]))
        assert abs(got[m, j] - want) <= gamma * scale + 1e-30, (case["tag"], m, j)


def test_packed_gemm_host_checks():
    with pytest.raises(ttc.TTCError) as ei:
        ttc.PackedGemm((0, 1), (64, 60), 1, 64)           # K = 60 is not a multiple of 8
    assert ei.value.name == "TTC_ERR_INVALID_SIZE"
    with pytest.raises(ttc.TTCError) as ei:
        ttc.PackedGemm((0, 1), (64, 64), 0, 64)
    assert ei.value.name == "TTC_ERR_INVALID_ARG"
    g = ttc.PackedGemm((0, 1), (64, 64), 1, 64)
    A = torch.zeros(64 * 64, device="cuda")
    B = torch.zeros(64 * 64, dtype=torch.int16, device="cuda")
    with pytest.raises(ttc.TTCError) as ei:
        g.execute(A, B, A)
    assert ei.value.name == "TTC_ERR_ALIAS"


def test_packed_gemm_wait_limit_reports_timeout_and_keeps_the_context():
    """Failure detection without a GPU fault: under the testing hook no MMA
    is committed, so the kernel's bounded mbarrier waits run out; it records
    the error word, frees its tensor memory and returns without writing C.
    The host reads TTC_ERR_TIMEOUT once, and the context keeps working."""
    g = ttc.PackedGemm((0, 1), (128, 192), 1, 256)           # one CTA, three k stages
    A = torch.ones(128 * 192, device="cuda")
    B = torch.zeros(192 * 256, dtype=torch.int16, device="cuda")
    C = torch.full((128 * 256,), 7.0, device="cuda")
    g.skip_mma(True)
    g.execute(A, B, C)
    torch.cuda.synchronize()
    with pytest.raises(ttc.TTCError) as ei:
        g.check()
    assert ei.value.name == "TTC_ERR_TIMEOUT"
    assert bool((C == 7.0).all())                             # C untouched
    g.check()                                                 # reported once
    g.skip_mma(False)
    g.execute(A, B, C)                                        # the same plan works again
    torch.cuda.synchronize()
    g.check()
    assert bool((C == 0.0).all())                             # Bm = 0
    run((0, 1), (128, 192), 1, 256, seed=7)                  # and a fresh plan matches the oracle


def run_fp8(perm, sizes, rank_m, n, alpha=1.0, outer=None, seed=0, identity=False):
    """E4M3 operands: P's codes against the oracle's FP8 permutation with the
    same scale (bit for bit, through an identity Bm) or C against the exact
    product of the decoded codes (random Bm codes)."""
    g = inputs.rng(seed)
    oa = outer or sizes
    A = g.normal(0, 1, int(np.prod(oa, dtype=np.int64))).astype(np.float32)
    gemm = ttc.PackedGemm(perm, sizes, rank_m, n, alpha, outer)
    inf = gemm.info()
    M, K = inf["m"], inf["k"]
    sp, _ = oracle.fp8_scale(sizes, A, alpha, oracle.F32, outer)
    sp = float(np.float32(sp))
    sb = 0.03125 if not identity else 1.0
    if identity:
        assert n == K
        Bcodes = np.zeros(K * n, np.uint8)
        Bcodes[np.arange(K) * (K + 1)] = oracle.e4m3_from_f32(np.ones(1, np.float32))[0]
    else:
        Bcodes = oracle.e4m3_from_f32(g.uniform(-1, 1, K * n).astype(np.float32))
    dsp = torch.tensor([sp], dtype=torch.float32, device="cuda")
    dsb = torch.tensor([sb], dtype=torch.float32, device="cuda")
    gemm.set_fp8(dsp, dsb)
    dA = torch.from_numpy(A).cuda()
    dB = torch.from_numpy(Bcodes).cuda()
    dC = torch.full((M * n,), float("nan"), device="cuda")
    gemm.execute(dA, dB, dC)
    torch.cuda.synchronize()
    gemm.check()
    got = dC.cpu().numpy().reshape(n, M).T
    sB = [sizes[p] for p in perm]
    Pc = np.zeros(int(np.prod(sB, dtype=np.int64)), np.uint8)
    oracle.permute(perm, sizes, A, Pc, alpha, 0.0, oracle.F32, oracle.E4M3, outer, None, fp8_scale=sp)
    P = oracle.e4m3_to_f32(Pc).astype(np.float64).reshape(K, M).T
    if identity:
        want = (np.float32(sp) * P.astype(np.float32))
        assert np.array_equal(got, want), (perm, sizes, int((got != want).sum()))
        return
    Bv = oracle.e4m3_to_f32(Bcodes).astype(np.float64).reshape(n, K).T
    s = np.float64(np.float32(np.float32(sp) * np.float32(sb)))
    want = s * (P @ Bv)
    scale = s * (np.abs(P) @ np.abs(Bv))
    u = 2.0 ** -23
    gamma = (K + 2) * u / (1 - (K + 2) * u)
    err = np.abs(got.astype(np.float64) - want)
    bad = ~(err <= gamma * scale + 1e-30)
    assert not bad.any(), (perm, sizes, int(bad.sum()), float(np.nanmax(err)))


@pytest.mark.parametrize("perm,sizes,rank_m,outer", [
    ((0, 1), (128, 64), 1, None),                # one tile, m dense in A (scalar pack)
    ((1, 0), (80, 200), 1, None),                # A stored K x M: k dense (16-byte pack loads)
    ((0, 1), (300, 144), 1, (320, 160)),         # a sub-block, ragged M
    ((0, 2, 1, 3), (20, 8, 13, 8), 2, None),     # the TTGT layout
])
def test_packed_gemm_fp8_codes_are_the_fp8_permutation(perm, sizes, rank_m, outer):
    sB = [sizes[p] for p in perm]
    K = int(np.prod(sB[rank_m:]))
    run_fp8(perm, sizes, rank_m, K, alpha=1.25, outer=outer, seed=11, identity=True)


@pytest.mark.parametrize("perm,sizes,rank_m,n,outer", [
    ((0, 1), (128, 64), 1, 256, None),
    ((1, 0), (160, 520), 1, 300, None),          # several k stages (128 per stage), ragged N
    ((0, 1), (300, 144), 1, 257, (320, 160)),
    ((0, 2, 1, 3), (20, 16, 13, 16), 2, 96, None),
])
def test_packed_gemm_fp8_product_within_bound(perm, sizes, rank_m, n, outer):
    run_fp8(perm, sizes, rank_m, n, alpha=-0.5, outer=outer, seed=12)


def test_packed_gemm_fp8_host_checks():
    g = ttc.PackedGemm((0, 1), (64, 24), 1, 64)          # K = 24: BF16 fine, E4M3 needs K % 16 == 0
    s = torch.ones(1, device="cuda")
    with pytest.raises(ttc.TTCError) as ei:
        g.set_fp8(s, s)
    assert ei.value.name == "TTC_ERR_INVALID_SIZE"
    g2 = ttc.PackedGemm((0, 1), (64, 32), 1, 64)
    with pytest.raises(ttc.TTCError) as ei:
        g2.set_fp8(s, None)
    assert ei.value.name == "TTC_ERR_INVALID_ARG"
