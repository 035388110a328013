"""GPU parity of the TTGT contractions (ttc_contraction_*) against the
oracle's definition, within the forward error bound of a dot product of
length K: |C - C_exact| <= gamma_(K+2) * (|alpha| |A||B| + |beta| |C|), with
gamma_n = n u / (1 - n u) and u the unit roundoff of the GEMM's accumulation
(2^-24 for FP32 and for BF16 operands, 2^-53 for FP64).  For BF16 GEMMs the
exact value is taken on the operands rounded to BF16 by the packing
transposes (round to nearest even).  The oracle evaluates in binary64, so for
FP64 data its own rounding error (the same bound) is added to the
tolerance."""
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


LAYOUTS = [
    ((0, 1), (1, 2), (0, 2)),                    # plain matrix product: no transpose
    ((1, 0), (2, 1), (2, 0)),                    # both operands transposed, C = [free B, free A]
    ((0, 3, 1, 4), (4, 2, 3), (2, 1, 0)),        # permuted operands, C transposed by the GEMM
    ((0, 3, 1, 4), (4, 2, 3), (1, 2, 0)),        # interleaved free labels: C through a workspace
    ((3, 0, 4, 1), (2, 4, 3), (0, 1, 2)),
    ((0, 1), (2, 3), (3, 0, 2, 1)),              # outer product (K = 1)
    ((5, 1, 0, 6), (6, 3, 1, 5), (3, 0)),        # three contracted labels
]


def run_case(ma, mb, mc, ext, dtype, gemm, alpha, beta, seed, variant=None, autotune=0):
    sa, sb, sc = (tuple(ext[m] for m in ms) for ms in (ma, mb, mc))
    npdt = np.float32 if dtype == "f32" else np.float64
    g = inputs.rng(seed)
    A = g.uniform(-1, 1, int(np.prod(sa, dtype=np.int64))).astype(npdt)
    B = g.uniform(-1, 1, int(np.prod(sb, dtype=np.int64))).astype(npdt)
    C0 = g.uniform(-1, 1, int(np.prod(sc, dtype=np.int64))).astype(npdt)
    con = ttc.Contraction(ma, sa, mb, sb, mc, sc, dtype, gemm, alpha, beta)
    if variant is not None:
        con.gemm_variant(variant)
    if autotune:
        con.autotune(autotune)
    dA, dB, dC = (torch.from_numpy(x.copy()).cuda() for x in (A, B, C0))
    con.execute(dA, dB, dC)
    torch.cuda.synchronize()
    if variant:
        assert con.gemm_variant() == variant
    got = dC.cpu().numpy().astype(np.float64)
    Ar, Br = A, B
    if gemm == "bf16":
        Ar = oracle.bf16_from_f32(A).astype(np.uint32).__lshift__(16).view(np.float32)
        Br = oracle.bf16_from_f32(B).astype(np.uint32).__lshift__(16).view(np.float32)
    want = oracle.contract(ma, Ar, sa, mb, Br, sb, mc, C0, sc, alpha, beta)
    scale = oracle.contract(ma, Ar, sa, mb, Br, sb, mc, C0, sc, alpha, beta, absolute=True)
    K = int(np.prod([ext[m] for m in set(ma) & set(mb)], dtype=np.int64)) if set(ma) & set(mb) else 1
    u = 2.0 ** -53 if dtype == "f64" else 2.0 ** -24
    n = K + 2
    gamma = n * u / (1 - n * u)
    if dtype == "f64":
        gamma *= 2      # the oracle evaluates in binary64 too: its own error has the same bound
    err = np.abs(got - want)
    tol = gamma * scale + (2.0 ** -149 if dtype == "f32" else 0.0)
    bad = err > tol
    assert not bad.any(), (ma, mb, mc, dtype, gemm, int(bad.sum()), float(err.max()), float(tol[bad][0]))
    return con


@pytest.mark.parametrize("dtype,gemm", [("f32", "f32"), ("f64", "f64"), ("f32", "bf16")])
@pytest.mark.parametrize("layout", range(len(LAYOUTS)))
def test_contraction_matches_definition(dtype, gemm, layout):
    ma, mb, mc = LAYOUTS[layout]
    g = inputs.rng(400 + layout)
    labels = set(ma) | set(mb) | set(mc)
    ext = {m: int(g.integers(3, 19)) for m in labels}
    for alpha, beta in ((1.0, 0.0), (0.75, -1.25)):
        run_case(ma, mb, mc, ext, dtype, gemm, alpha, beta, 500 + layout)


@pytest.mark.parametrize("layout", [((0, 3, 1, 4), (4, 2, 3), (2, 1, 0)),
                                    ((0, 4, 1, 5), (5, 2, 4, 3), (0, 1, 2, 3)),
                                    ((5, 1, 0, 6), (6, 3, 1, 5), (3, 0))])
def test_autotuned_bf16_contraction_matches_definition(layout):
    """The BF16 mode's autotuner also tries the contracted labels in B's
    order (these layouts order them differently in A and B) and keeps the
    faster pair of operand permutes; either way the result is the
    definition's."""
    ma, mb, mc = layout
    g = inputs.rng(900)
    ext = {m: int(g.integers(5, 17)) for m in set(ma) | set(mb) | set(mc)}
    for alpha, beta in ((1.0, 0.0), (0.75, -1.25)):
        run_case(ma, mb, mc, ext, "f32", "bf16", alpha, beta, 910, autotune=8)


def test_contraction_larger_ragged_and_degenerate():
    # several GEMM tiles with ragged edges, and a case for each layout kind
    run_case((0, 3, 1, 4), (4, 2, 3), (1, 2, 0), {0: 37, 1: 29, 2: 71, 3: 13, 4: 11}, "f32", "f32", 1.3, 0.5, 7)
    run_case((0, 3, 1, 4), (4, 2, 3), (2, 1, 0), {0: 37, 1: 29, 2: 71, 3: 13, 4: 11}, "f32", "bf16", 1.3, 0.0, 8)
    run_case((0, 1), (1, 2), (0, 2), {0: 257, 1: 129, 2: 65}, "f64", "f64", -0.5, 2.0, 9)
    # an empty contracted extent leaves beta * C
    run_case((0, 1), (1, 2), (2, 0), {0: 5, 1: 0, 2: 6}, "f32", "f32", 1.0, 0.5, 10)
    # an empty free extent is a no-op
    con = ttc.Contraction((0, 1), (0, 4), (1, 2), (4, 3), (0, 2), (0, 3))
    con.execute(0, 0, 0)


def test_contraction_rejects_overlap_and_reuses_workspace():
    ext = {0: 20, 1: 30, 2: 10, 3: 7}
    con = run_case((0, 3, 1), (3, 2), (1, 2, 0), ext, "f32", "f32", 1.0, 0.0, 11)
    A = torch.zeros(20 * 7 * 30, device="cuda")
    B = torch.zeros(7 * 10, device="cuda")
    with pytest.raises(ttc.TTCError) as ei:
        con.execute(A, B, A)
    assert ei.value.name == "TTC_ERR_ALIAS"
    # the same plan on new data (workspaces kept from the first execution)
    run_case((0, 3, 1), (3, 2), (1, 2, 0), ext, "f32", "f32", 1.0, 0.0, 12)


@pytest.mark.parametrize("case", range(3))
def test_full_size_contraction_sampled(case):
    """The bench's contractions at full size: sampled entries of C against the
    definition, each a dot product of length K computed on the host."""
    from paper_1607_01249_gb300.inputs import contraction_cases
    c = contraction_cases()[case]
    ma, mb, mc, ext = c["modes_a"], c["modes_b"], c["modes_c"], c["extents"]
    sa, sb, sc = (tuple(ext[m] for m in ms) for ms in (ma, mb, mc))
    g = inputs.rng(600 + case)
    A = g.uniform(-1, 1, int(np.prod(sa, dtype=np.int64))).astype(np.float32)
    B = g.uniform(-1, 1, int(np.prod(sb, dtype=np.int64))).astype(np.float32)
    con = ttc.Contraction(ma, sa, mb, sb, mc, sc, "f32", "f32", 1.0, 0.0)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dC = torch.zeros(int(np.prod(sc, dtype=np.int64)), device="cuda")
    con.execute(dA, dB, dC)
    torch.cuda.synchronize()
    got = dC.cpu().numpy()
    a = A.reshape(sa, order="F").astype(np.float64)
    b = B.reshape(sb, order="F").astype(np.float64)
    contracted = [m for m in ma if m in mb]
    for _ in range(64):
        idx = {m: int(g.integers(0, ext[m])) for m in mc}
        sl_a = tuple(idx[m] if m in idx else slice(None) for m in ma)
        sl_b = tuple(idx[m] if m in idx else slice(None) for m in mb)
        # the remaining axes of a and b are the contracted labels, in each operand's order
        ra = [m for m in ma if m not in idx]
        rb = [m for m in mb if m not in idx]
        va = np.transpose(a[sl_a], [ra.index(m) for m in contracted])
        vb = np.transpose(b[sl_b], [rb.index(m) for m in contracted])
        exact = float(np.sum(va * vb))
        scale = float(np.sum(np.abs(va) * np.abs(vb)))
        off, st = 0, 1
        for m, s in zip(mc, sc):
            off += idx[m] * st
            st *= s
        K = int(np.prod([ext[m] for m in contracted]))
        n = K + 2
        assert abs(float(got[off]) - exact) <= n * 2.0 ** -24 / (1 - n * 2.0 ** -24) * scale


@pytest.mark.parametrize("variant", [1, 2, 3, 4, 5, 6])
def test_bf16_gemm_tiles_and_edges(variant):
    """The tensor-core GEMM of the BF16 mode in each tile shape (one CTA per
    128 x 256, 128 x 192 or 128 x 128 tile; a CTA pair per 256 x 256 or
    256 x 128 tile) over several
    tiles in both directions, ragged M, N and K (K a multiple of 8 and not,
    so that the operands' row pitch is padded), M within one CTA's half of a
    pair tile, with beta, and with C taking the GEMM's output directly,
    transposed, and through a workspace."""
    for ext, mc, beta in (({0: 300, 1: 1000, 2: 600}, (0, 2), 0.5),      # M, N ragged; K % 64 != 0
                          ({0: 129, 1: 77, 2: 257}, (2, 0), 0.0),        # K % 8 != 0: padded pitch
                          ({0: 40, 1: 8, 2: 30}, (0, 2), -1.0),          # one K stage, M < 128
                          ({0: 520, 1: 4100, 2: 1030}, (0, 2), 0.0)):    # many K stages, ragged pair tiles
        run_case((0, 1), (1, 2), mc, ext, "f32", "bf16", 1.25, beta, 20, variant)
    run_case((0, 3, 1, 4), (4, 2, 3), (1, 2, 0), {0: 37, 1: 29, 2: 71, 3: 13, 4: 11}, "f32", "bf16", 1.3, 0.5, 21,
             variant)
    con = run_case((5, 1, 0, 6), (6, 3, 1, 5), (3, 0), {0: 150, 1: 5, 3: 270, 5: 7, 6: 9}, "f32", "bf16", 1.0,
                   0.0, 22, variant)
    con.check()


def test_bf16_gemm_matches_cublas_on_the_same_operands():
    """The same K-major BF16 operands through cuBLAS (the timed comparison):
    both within the dot-product bound of the definition, and of each other."""
    ext = {0: 260, 1: 520, 2: 390}
    ours = run_case((0, 1), (1, 2), (0, 2), ext, "f32", "bf16", 1.0, 0.25, 23)
    g = inputs.rng(23)
    sa, sb, sc = (260, 520), (520, 390), (260, 390)
    A = g.uniform(-1, 1, 260 * 520).astype(np.float32)
    B = g.uniform(-1, 1, 520 * 390).astype(np.float32)
    C0 = g.uniform(-1, 1, 260 * 390).astype(np.float32)
    outs = []
    for use in (False, True):
        con = ttc.Contraction((0, 1), sa, (1, 2), sb, (0, 2), sc, "f32", "bf16", 1.0, 0.25).use_cublas(use)
        dA, dB, dC = (torch.from_numpy(x.copy()).cuda() for x in (A, B, C0))
        con.execute(dA, dB, dC)
        torch.cuda.synchronize()
        outs.append(dC.cpu().numpy().astype(np.float64))
    scale = np.abs(A.reshape(sa, order="F")).astype(np.float64) @ np.abs(B.reshape(sb, order="F")).astype(np.float64)
    n = 520 + 2
    tol = 2 * n * 2.0 ** -24 / (1 - n * 2.0 ** -24) * (scale.ravel(order="F") + 0.25 * np.abs(C0))
    assert np.all(np.abs(outs[0] - outs[1]) <= tol)
    ours.check()


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("case", range(3))
def test_full_size_bf16_contraction_sampled(case, variant):
    """The bench's contractions at full size in the BF16 mode, in the tile
    shape the library picks and in each forced one: sampled entries of C
    against the definition on the operands rounded to BF16."""
    from paper_1607_01249_gb300.inputs import contraction_cases
    c = contraction_cases()[case]
    ma, mb, mc, ext = c["modes_a"], c["modes_b"], c["modes_c"], c["extents"]
    sa, sb, sc = (tuple(ext[m] for m in ms) for ms in (ma, mb, mc))
    g = inputs.rng(700 + case)
    A = g.uniform(-1, 1, int(np.prod(sa, dtype=np.int64))).astype(np.float32)
    B = g.uniform(-1, 1, int(np.prod(sb, dtype=np.int64))).astype(np.float32)
    con = ttc.Contraction(ma, sa, mb, sb, mc, sc, "f32", "bf16", 1.0, 0.0)
    con.gemm_variant(variant)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dC = torch.zeros(int(np.prod(sc, dtype=np.int64)), device="cuda")
    con.execute(dA, dB, dC)
    torch.cuda.synchronize()
    con.check()
    assert con.gemm_variant() == variant or (variant == 0 and con.gemm_variant() in (1, 2, 3, 4, 5, 6))
    got = dC.cpu().numpy()
    Ar = oracle.bf16_from_f32(A).astype(np.uint32).__lshift__(16).view(np.float32)
    Br = oracle.bf16_from_f32(B).astype(np.uint32).__lshift__(16).view(np.float32)
    a = Ar.reshape(sa, order="F").astype(np.float64)
    b = Br.reshape(sb, order="F").astype(np.float64)
    contracted = [m for m in ma if m in mb]
    K = int(np.prod([ext[m] for m in contracted]))
    n = K + 2
    for _ in range(64):
        idx = {m: int(g.integers(0, ext[m])) for m in mc}
        sl_a = tuple(idx[m] if m in idx else slice(None) for m in ma)
        sl_b = tuple(idx[m] if m in idx else slice(None) for m in mb)
        ra = [m for m in ma if m not in idx]
        rb = [m for m in mb if m not in idx]
        va = np.transpose(a[sl_a], [ra.index(m) for m in contracted])
        vb = np.transpose(b[sl_b], [rb.index(m) for m in contracted])
        exact = float(np.sum(va * vb))
        scale = float(np.sum(np.abs(va) * np.abs(vb)))
        off, st = 0, 1
        for m, s in zip(mc, sc):
            off += idx[m] * st
            st *= s
        assert abs(float(got[off]) - exact) <= n * 2.0 ** -24 / (1 - n * 2.0 ** -24) * scale
