"""GPU parity: libttc (sm_103a kernels, through the C ABI) against the CPU
oracle, element by element, on seeded inputs.

Bar: bit-exact against the oracle's rounding sequence for every dtype (NaN
payloads only for pure bit copies), and within the stated tolerance of the
exact value (2 FP32 ulps for FP32 data, 1e-15 relative for FP64 data, 1 BF16
ulp for BF16 output, all at the scale max(|alpha a|, |beta b|, |r|)).
"""
import itertools

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1607_01249_gb300 import build as ttc_build
from paper_1607_01249_gb300 import inputs
from paper_1607_01249_gb300 import ttc
from tests import gpu_helpers as H
from paper_1607_01249_gb300.inputs import Problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    ttc_build.build()
    ttc.lib()


def small_sweep(Ns=(2, 3, 4, 5, 6), target=1 << 15, perms=4, seed=11):
    g = inputs.rng(seed)
    out = []
    for N in Ns:
        for perm in inputs.sweep_perms(N, g, perms):
            out.append((perm, inputs.near_equal_sizes(N, target, g, tol=0.05)))
    return out


SMALL = small_sweep()


def test_single_4d_workload():
    p = inputs.single_4d()
    H.full_check(p, seed=0)


@pytest.mark.parametrize("dt", ["f32", "f64"])
@pytest.mark.parametrize("beta", [0.0, 0.4])
@pytest.mark.parametrize("case", range(len(SMALL)))
def test_small_sweep(case, dt, beta):
    perm, sizes = SMALL[case]
    p = Problem(perm=perm, sizes=sizes, dtype_in=dt, dtype_out=dt, alpha=1.7, beta=beta)
    H.full_check(p, seed=case)


PAIRS = [("f32", "f32"), ("f32", "f64"), ("f32", "bf16"), ("f32", "e4m3"), ("f64", "f64"), ("f64", "f32"),
         ("bf16", "bf16"), ("bf16", "f32"), ("bf16", "e4m3")]


@pytest.mark.parametrize("din,dout", PAIRS)
@pytest.mark.parametrize("ab", [(1.0, 0.0), (1.7, 0.0), (-0.75, 0.4)])
@pytest.mark.parametrize("shape", [((2, 0, 3, 1), (33, 17, 20, 9)), ((0, 2, 1), (300, 21, 13)),
                                   ((0, 2, 1), (7, 61, 40)), ((1, 0), (1000, 3))])
def test_dtype_pairs(din, dout, ab, shape):
    alpha, beta = ab
    if dout == "e4m3" and beta != 0.0:
        pytest.skip("FP8 output is beta == 0 only")
    perm, sizes = shape
    p = Problem(perm=perm, sizes=sizes, dtype_in=din, dtype_out=dout, alpha=alpha, beta=beta)
    H.full_check(p, seed=3, dist="normal")


@pytest.mark.parametrize("trial", range(12))
def test_outer_sizes_and_canaries(trial):
    g = inputs.rng(200 + trial)
    N = int(g.integers(2, 6))
    perm = inputs.random_perm(N, g)
    sizes = tuple(int(x) for x in g.integers(2, 40 if N < 4 else 14, size=N))
    oa = tuple(s + int(g.integers(0, 5)) for s in sizes)
    sb = tuple(sizes[q] for q in perm)
    ob = tuple(s + int(g.integers(0, 5)) for s in sb) if trial % 2 else None
    dt = ["f32", "f64", "bf16"][trial % 3]
    beta = 0.0 if trial % 4 < 2 else 0.5
    p = Problem(perm=perm, sizes=sizes, dtype_in=dt, dtype_out=dt, alpha=1.25, beta=beta, outer_a=oa,
                outer_b=ob)
    H.full_check(p, seed=trial)   # whole B buffer compared: elements outside the sub-tensor unchanged


@pytest.mark.parametrize("case", inputs.packing_cases(), ids=lambda c: f"{c.tag}-{c.dtype_out}")
def test_packing_workloads(case):
    if case.tag.startswith("panel"):
        M, K = case.extra["matrix"]
        m0, k0 = case.extra["offset"]
        full = inputs.tensor_for("f32", M * K, 5, "normal")
        A = full[m0 + k0 * M:]              # A points at the sub-block's first element
        B0 = np.zeros(case.vol_b, inputs.STORAGE[case.dtype_out])
        got, scale = H.run_gpu(case, A, B0)
        want, oscale = H.oracle_mirror(case, A, B0)
    else:
        A, B0 = H.make_inputs(case, 6, "normal")
        got, scale = H.run_gpu(case, A, B0)
        want, oscale = H.oracle_mirror(case, A, B0)
    if case.dtype_out == "e4m3":
        assert scale == oscale
        rep = H.fp8_error_report(case, A, got, scale)
        assert rep["bound_ok"], rep
    ok, msg = H.compare_bits(got, want, case.dtype_out, nan_as_nan=True)
    assert ok, msg
    ok, msg = H.tolerance_check(case, A, B0, got)
    assert ok, msg


def test_fp8_caller_scale_and_degenerate_amax():
    p = Problem(perm=(1, 0), sizes=(96, 70), dtype_in="f32", dtype_out="e4m3")
    A, B0 = H.make_inputs(p, 7, "normal")
    s = torch.tensor([0.01], dtype=torch.float32, device="cuda")
    got, scale = H.run_gpu(p, A, B0, scale_dev=s)
    assert scale == np.float32(0.01)
    want, _ = H.oracle_mirror(p, A, B0, scale=float(np.float32(0.01)))
    assert np.array_equal(got, want)
    Z = Problem(perm=(1, 0), sizes=(96, 70), dtype_in="f32", dtype_out="e4m3")
    A0 = np.zeros(Z.vol_a, np.float32)
    got, scale = H.run_gpu(Z, A0, np.zeros(Z.vol_b, np.uint8))
    assert scale == 1.0 and not got.any()


@pytest.mark.parametrize("scale", [0.01, 0.7, 3.0, 0.25, 1.0e-6])
def test_fp8_codes_at_and_around_rounding_boundaries(scale):
    """FP8 codes of quotients at every E4M3 rounding boundary (the midpoints
    between neighbouring codes, the subnormal ones included) and a few
    binary32 ulps on either side, for several caller scales: the kernels'
    reciprocal fast path must fall back to the exact division exactly where
    it matters, so the codes equal the oracle's bit for bit."""
    s32 = np.float32(scale)
    codes = np.arange(0, 0x7F, dtype=np.uint8)                  # finite non-negative codes
    vals = oracle.e4m3_to_f32(codes).astype(np.float64)
    mids = (vals[:-1] + vals[1:]) / 2                              # exact in binary32
    q = np.concatenate([mids, vals]).astype(np.float32)
    steps = np.arange(-6, 7, dtype=np.int64)
    qq = (q.view(np.int32)[:, None] + steps[None, :]).astype(np.int32).view(np.float32).ravel()
    qq = qq[np.isfinite(qq) & (qq >= 0)]
    a = np.concatenate([qq, -qq]).astype(np.float64) * np.float64(s32)   # alpha * a / scale ~ the quotients
    A = a.astype(np.float32)
    n = A.size
    p = Problem(perm=(1, 0), sizes=(n // 2, 2), dtype_in="f32", dtype_out="e4m3")
    dev_scale = torch.tensor([float(s32)], dtype=torch.float32, device="cuda")
    got, sc = H.run_gpu(p, A, np.zeros(n, np.uint8), scale_dev=dev_scale)
    assert sc == s32
    want, _ = H.oracle_mirror(p, A, np.zeros(n, np.uint8), scale=float(s32))
    ok, msg = H.compare_bits(got, want, "e4m3", nan_as_nan=True)
    assert ok, msg


def test_beta_zero_never_reads_B():
    for dt in ("f32", "f64", "bf16"):
        for perm, sizes in [((2, 0, 1), (40, 30, 20)), ((0, 2, 1), (200, 10, 30))]:
            p = Problem(perm=perm, sizes=sizes, dtype_in=dt, dtype_out=dt, alpha=1.7, beta=0.0)
            fill = {"f32": np.float32(np.nan), "f64": np.nan, "bf16": np.uint16(0x7FC1)}[dt]
            A, B0, got, _ = H.full_check(p, seed=9, b_fill=fill)
            assert not np.isnan(H.as_float(got, dt)).any()


def test_bitcopy_special_patterns():
    pats32 = np.array([0x80000000, 0x00000001, 0x807FFFFF, 0x7FC00123, 0xFFA00001, 0x7F800000, 0xFF800000,
                       0x00800000, 0x7F7FFFFF, 0x3F800000], np.uint32)
    for perm, sizes in [((1, 0), (50, 37)), ((0, 2, 1), (64, 5, 7)), ((2, 1, 0), (9, 10, 11))]:
        n = int(np.prod(sizes))
        A = np.resize(pats32, n).view(np.float32)
        p = Problem(perm=perm, sizes=sizes)
        got, _ = H.run_gpu(p, A, np.zeros(n, np.float32))
        want, _ = H.oracle_mirror(p, A, np.zeros(n, np.float32))
        assert got.tobytes() == want.tobytes()
        A64 = np.resize(np.array([0x8000000000000000, 1, 0x7FF8000000000123, 0xFFF0000000000001], np.uint64),
                        n).view(np.float64)
        p64 = Problem(perm=perm, sizes=sizes, dtype_in="f64", dtype_out="f64")
        got, _ = H.run_gpu(p64, A64, np.zeros(n, np.float64))
        want, _ = H.oracle_mirror(p64, A64, np.zeros(n, np.float64))
        assert got.tobytes() == want.tobytes()
        A16 = np.resize(np.array([0x8000, 0x0001, 0x7FC3, 0xFF81, 0x7F80], np.uint16), n)
        p16 = Problem(perm=perm, sizes=sizes, dtype_in="bf16", dtype_out="bf16")
        got, _ = H.run_gpu(p16, A16, np.zeros(n, np.uint16))
        want, _ = H.oracle_mirror(p16, A16, np.zeros(n, np.uint16))
        assert got.tobytes() == want.tobytes()


@pytest.mark.parametrize("perm,sizes", [((0,), (1,)), ((0,), (1000003,)), ((1, 0), (1, 1)),
                                        ((2, 1, 0), (1, 1, 7)), ((1, 0, 2), (1, 5, 1)),
                                        (tuple(range(15, -1, -1)), (2,) * 16),
                                        ((3, 1, 0, 2), (2, 3, 1, 4)), ((1, 0), (3, 100003))])
def test_edge_shapes(perm, sizes):
    for dt, beta in (("f32", 0.0), ("f64", 0.5)):
        p = Problem(perm=perm, sizes=sizes, dtype_in=dt, dtype_out=dt, alpha=1.7, beta=beta)
        H.full_check(p, seed=4)


def test_empty_problem_launches_nothing():
    p = ttc.Plan((1, 0), (0, 7))
    before = ttc.launch_count()
    p.execute(torch.empty(0, device="cuda"), torch.empty(0, device="cuda"))
    assert ttc.launch_count() == before


def test_every_candidate_schedule_agrees():
    for perm, sizes in [SMALL[3], SMALL[9], SMALL[15], ((2, 0, 3, 1), (32, 40, 24, 36))]:
        p = Problem(perm=perm, sizes=sizes, alpha=1.7, beta=0.4)
        plan = ttc.Plan(p.perm, p.sizes, alpha=p.alpha, beta=p.beta)
        A, B0 = H.make_inputs(p, 1)
        want, _ = H.oracle_mirror(p, A, B0)
        for i in range(plan.info()["ncandidates"]):
            plan.select(i)
            got, _ = H.run_gpu(p, A, B0, plan=plan)
            ok, msg = H.compare_bits(got, want, "f32", nan_as_nan=True)
            assert ok, (i, msg)


TMA_CASES = [
    ((64, 96), "f32", "f32", 1.0, 0.0, None),
    ((100, 36), "f32", "bf16", 1.5, 0.0, None),
    ((1000, 333), "f64", "f32", 0.75, 0.5, None),
    ((96, 130), "f64", "f64", 1.25, -0.5, None),
    ((200, 260), "f32", "e4m3", 1.0, 0.0, None),
    ((4, 2000), "f32", "f32", -2.0, 0.25, None),       # fewer rows than a box
    ((2048, 20), "f32", "f64", 1.0, 0.0, None),        # fewer columns than a box
    ((120, 70), "f32", "f32", 1.7, 0.4, (128, 75)),    # a sub-matrix (outer sizes)
]


@pytest.mark.parametrize("sizes,din,dout,alpha,beta,outer", TMA_CASES)
def test_tma_tile_matches_oracle(sizes, din, dout, alpha, beta, outer):
    """The TMA-staged tile of two swapped indices (boxes copied by the tensor
    memory accelerator, ragged edges zero-filled and masked) against the
    oracle, bit for bit, for each dtype pair it serves, with and without
    beta, and on a sub-matrix."""
    p = Problem(perm=(1, 0), sizes=sizes, dtype_in=din, dtype_out=dout, alpha=alpha, beta=beta, outer_a=outer,
                outer_b=tuple(reversed(outer)) if outer else None)
    plan = ttc.Plan(p.perm, p.sizes, p.dtype_in, p.dtype_out, p.alpha, p.beta, p.outer_a, p.outer_b)
    idx = [i for i in range(plan.info()["ncandidates"]) if "tma2d" in plan.describe(i)]
    assert idx, "the TMA tile should be a candidate here"
    plan.select(idx[0])
    assert plan.info()["kernel"] == "tma2d_kernel"
    assert plan.verify_schedule() == ""
    A, B0 = H.make_inputs(p, 31)
    got, _ = H.run_gpu(p, A, B0, plan=plan)
    want, _ = H.oracle_mirror(p, A, B0)
    ok, msg = H.compare_bits(got, want, dout, nan_as_nan=True)
    assert ok, msg


def test_tma_tile_reads_a_misaligned_a_directly():
    """A base address that is not 16-byte aligned cannot be described by a
    tensor map: the kernel then reads A directly, with the same results."""
    p = Problem(perm=(1, 0), sizes=(64, 50), dtype_in="f32", dtype_out="f32", alpha=1.3, beta=0.0)
    plan = ttc.Plan(p.perm, p.sizes, "f32", "f32", 1.3, 0.0)
    idx = [i for i in range(plan.info()["ncandidates"]) if "tma2d" in plan.describe(i)]
    plan.select(idx[0])
    A, B0 = H.make_inputs(p, 32)
    dA = torch.zeros(A.size + 1, dtype=torch.float32, device="cuda")
    dA[1:] = torch.from_numpy(A).cuda()
    dB = torch.from_numpy(B0.copy()).cuda()
    assert (dA[1:].data_ptr() % 16) != 0
    plan.execute(dA[1:], dB)
    torch.cuda.synchronize()
    want, _ = H.oracle_mirror(p, A, B0)
    ok, msg = H.compare_bits(dB.cpu().numpy(), want, "f32", nan_as_nan=True)
    assert ok, msg


def test_autotune_keeps_results_and_uses_no_user_memory():
    p = Problem(perm=(2, 0, 3, 1), sizes=(32, 40, 24, 36), alpha=1.7, beta=0.4)
    plan = ttc.Plan(p.perm, p.sizes, alpha=p.alpha, beta=p.beta)
    ms = plan.autotune(max_candidates=6)
    assert ms > 0
    H.full_check(p, seed=2, plan=plan)


def test_non_default_stream():
    p = Problem(perm=(1, 2, 0), sizes=(70, 80, 90), alpha=1.7, beta=0.4)
    A, B0 = H.make_inputs(p, 8)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        got, _ = H.run_gpu(p, A, B0, stream=s)
    want, _ = H.oracle_mirror(p, A, B0)
    ok, msg = H.compare_bits(got, want, "f32", True)
    assert ok, msg


# ---- full-size cases of the 2D..6D sweep (2^26 elements), whole output compared

FULL = [c for c in inputs.sweep_cases() if c.beta == 0.4 and
        ((c.dtype_in == "f32" and c.tag.endswith("p1")) or (c.dtype_in == "f64" and c.tag in ("N4p0", "N6p1")))]


@pytest.mark.slow
@pytest.mark.parametrize("case", FULL, ids=lambda c: f"{c.tag}-{c.dtype_in}")
def test_full_size_sweep_case(case):
    H.full_check(case, seed=1)


def test_many_schedules_in_one_process():
    """All candidate schedules of many shapes, back to back in one process (the
    launcher's per-kernel shared-memory limits must follow every size seen)."""
    g = inputs.rng(77)
    for trial in range(24):
        N = int(g.integers(2, 6))
        perm = inputs.random_perm(N, g)
        sizes = inputs.near_equal_sizes(N, int(2 ** g.uniform(12, 16)), g, tol=0.3)
        dt = ("f32", "f64")[trial % 2]
        p = Problem(perm=perm, sizes=sizes, dtype_in=dt, dtype_out=dt, alpha=1.5, beta=0.25 * (trial % 3))
        plan = ttc.Plan(p.perm, p.sizes, p.dtype_in, p.dtype_out, p.alpha, p.beta)
        A, B0 = H.make_inputs(p, trial)
        want, _ = H.oracle_mirror(p, A, B0)
        order = list(range(plan.info()["ncandidates"]))
        if trial % 2:
            order.reverse()
        for i in order:
            plan.select(i)
            got, _ = H.run_gpu(p, A, B0, plan=plan)
            ok, msg = H.compare_bits(got, want, dt, True)
            assert ok, (perm, sizes, i, msg)


def test_slot_table_tiles_every_pair_with_ragged_edges():
    """tile_slots_kernel schedules (tables ordered by address, masked edge
    tiles) for every dtype pair, with outer sizes and tails that leave most
    tiles at the tensor's edge cut short."""
    shapes = [((1, 0, 2), (37, 29, 11)), ((2, 0, 3, 1), (9, 23, 7, 13)), ((4, 2, 0, 3, 1), (5, 6, 7, 3, 9)),
              ((0, 2, 1), (13, 41, 17))]
    tried = 0
    for si, (perm, sizes) in enumerate(shapes):
        for din, dout in PAIRS:
            beta = 0.0 if dout == "e4m3" else 0.3
            oa = tuple(s + (si % 3) for s in sizes)
            p = Problem(perm=perm, sizes=sizes, dtype_in=din, dtype_out=dout, alpha=1.25, beta=beta, outer_a=oa)
            plan = ttc.Plan(p.perm, p.sizes, p.dtype_in, p.dtype_out, p.alpha, p.beta, p.outer_a, p.outer_b)
            A, B0 = H.make_inputs(p, 60 + si, "normal")
            want, wscale = H.oracle_mirror(p, A, B0)
            for i in range(plan.info()["ncandidates"]):
                plan.select(i)
                if not plan.info()["slot_tables"]:
                    continue
                got, scale = H.run_gpu(p, A, B0, plan=plan)
                if dout == "e4m3":
                    assert scale == wscale, (perm, sizes, din, dout, i)
                ok, msg = H.compare_bits(got, want, dout, nan_as_nan=True)
                assert ok, (perm, sizes, din, dout, i, msg)
                tried += 1
    assert tried >= 20


def test_fp8_plan_executed_repeatedly_tracks_each_inputs_scale():
    """Executions of one FP8 plan alternate between two amax words (each
    execution clears the other's): every execution's scale and codes must
    follow its own input, whatever the previous inputs were."""
    for din in ("f32", "bf16"):
        p = Problem(perm=(2, 0, 1), sizes=(67, 45, 33), dtype_in=din, dtype_out="e4m3", alpha=1.3)
        plan = ttc.Plan(p.perm, p.sizes, p.dtype_in, p.dtype_out, p.alpha, p.beta)
        for rep, mag in enumerate((1.0, 1e-3, 50.0, 50.0, 2.0, 1e-3)):
            A, B0 = H.make_inputs(p, 900 + rep, "normal")
            if din == "f32":
                A = (A * np.float32(mag)).astype(np.float32)
            else:
                A = inputs.bf16_bits_from_f32_trunc(H.as_float(A, "bf16").astype(np.float32) * np.float32(mag))
            got, scale = H.run_gpu(p, A, B0, plan=plan)
            want, wscale = H.oracle_mirror(p, A, B0)
            assert scale == wscale, (din, rep, scale, wscale)
            ok, msg = H.compare_bits(got, want, "e4m3", nan_as_nan=True)
            assert ok, (din, rep, msg)


def test_autotune_choice_is_remembered_for_new_plans(tmp_path):
    """A later plan of the same problem starts from the autotuner's choice
    (process-wide cache), and the cache survives a save/load."""
    p = Problem(perm=(1, 0), sizes=(3000, 2000), alpha=1.3)
    a = ttc.Plan(p.perm, p.sizes, alpha=p.alpha)
    a.autotune(max_candidates=8)
    chosen = a.info()["candidate"]
    path = str(tmp_path / "tune.txt")
    ttc.tune_cache_save(path)
    assert any(line.strip() for line in open(path))
    ttc.tune_cache_load(path)
    b = ttc.Plan(p.perm, p.sizes, alpha=p.alpha)
    H.full_check(p, seed=3, plan=b)              # first execution applies the cache
    assert a.describe(chosen).split(" est_us")[0] == b.describe().split(" est_us")[0]


ROWVEC_CASES = [
    ((0, 2, 1), (256, 16, 64), "f32", "bf16", 1.0, 0.0),
    ((0, 2, 1), (36, 10, 7), "f32", "f32", 1.5, 0.5),
    ((0, 2, 1), (64, 30, 20), "f64", "f64", -0.75, 0.25),
    ((0, 2, 1, 3), (64, 8, 12, 5), "bf16", "f32", 1.0, 0.5),
    ((0, 2, 1), (128, 9, 40), "f32", "e4m3", 1.0, 0.0),
    ((0, 2, 1), (370, 37, 48), "f64", "f64", 1.7, 0.4),   # a tile wider than the element-wise copy's
]


@pytest.mark.parametrize("perm,sizes,din,dout,alpha,beta", ROWVEC_CASES)
def test_vector_row_copy_matches_oracle(perm, sizes, din, dout, alpha, beta):
    """The multi-row copy with 16-byte accesses (every candidate of that
    kind) against the oracle, bit for bit, with aligned bases and with A and
    B offset by one element (element accesses, the same walk)."""
    p = Problem(perm=perm, sizes=sizes, dtype_in=din, dtype_out=dout, alpha=alpha, beta=beta)
    plan = ttc.Plan(p.perm, p.sizes, p.dtype_in, p.dtype_out, p.alpha, p.beta)
    idx = [i for i in range(plan.info()["ncandidates"])
           if "rows vec=" in plan.describe(i)]
    assert idx, "a vector row copy should be a candidate here"
    A, B0 = H.make_inputs(p, 33)
    want, _ = H.oracle_mirror(p, A, B0)
    for i in idx:
        plan.select(i)
        assert plan.info()["kernel"] == "rowcopy_vec_kernel"
        assert plan.verify_schedule() == ""
        got, _ = H.run_gpu(p, A, B0, plan=plan)
        ok, msg = H.compare_bits(got, want, dout, nan_as_nan=True)
        assert ok, (i, msg)
        # misaligned bases: one element past a fresh allocation
        dA = H.to_device(np.concatenate([A[:1], A]), din)[1:]
        dB = H.to_device(np.concatenate([B0[:1], B0]), dout)[1:]
        plan.execute(dA, dB)
        torch.cuda.synchronize()
        ok, msg = H.compare_bits(H.to_host(dB, dout), want, dout, nan_as_nan=True)
        assert ok, (i, "misaligned", msg)
