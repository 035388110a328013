"""The allocation-free entry point, ttc_execute_noalloc, against the oracle
and against ttc_execute.

Some callers cannot allocate device memory: their device memory belongs to a
pool allocator (a framework's caching allocator, a serving process with a
fixed budget), or they must not make the implicitly synchronising
cudaMalloc/cudaFree calls.  For them ttc_execute_noalloc runs the same
kernels with the scratch (FP8 amax/scale words, tile offset tables) in one
static device array of the library.  This file checks, through the C ABI,
that two calls in a row give the oracle's result and exactly what the
regular entry point gives (the array keeps the last call's contents between
calls), that a call on a fresh plan leaves the device's free memory as it
was, that calls of two plans on two streams ordered by an event give each
plan's result, and that a schedule needing more scratch than the array holds
is refused with a clear error.

The file is named so that pytest collects it last: should one of its checks
fail, a run that stops at the first failure has already run every other
test.  Its tests do not depend on that order.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1607_01249_gb300 import build as ttc_build
from paper_1607_01249_gb300 import inputs
from paper_1607_01249_gb300 import ttc
from paper_1607_01249_gb300.inputs import Problem
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu

STATIC_SCRATCH_BYTES = 8192   # TTC_NOALLOC_SCRATCH_BYTES in include/ttc.h


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    ttc_build.build()
    ttc.lib()


CASES = [
    # FP8 output with the scale computed on the device (amax word in the scratch)
    Problem(perm=(1, 3, 0, 2), sizes=(48, 64, 40, 56), dtype_in="f32", dtype_out="e4m3",
            outer_a=(64, 80, 48, 64), tag="fp8-sub4d"),
    Problem(perm=(2, 0, 1), sizes=(70, 33, 41), dtype_in="bf16", dtype_out="e4m3", tag="fp8-bf16"),
    # small indices: multi-index tile groups with offset tables in the scratch
    Problem(perm=(0, 5, 1, 2, 4, 3), sizes=(6, 7, 5, 6, 5, 7), alpha=1.7, beta=0.4, tag="6d-small"),
    Problem(perm=(2, 0, 3, 1), sizes=(17, 15, 15, 17), alpha=-0.5, beta=0.25, tag="4d-small"),
    # plain tile and streaming copy
    Problem(perm=(1, 0), sizes=(300, 257), dtype_in="f64", dtype_out="f64", alpha=1.7, beta=0.4, tag="2d-f64"),
    Problem(perm=(0, 2, 1), sizes=(130, 9, 11), dtype_in="bf16", dtype_out="bf16", alpha=1.7, beta=0.5,
            tag="copy-bf16"),
]


def fitting_plan(p: Problem):
    """A plan of p whose selected schedule fits the static scratch."""
    plan = ttc.Plan(p.perm, p.sizes, p.dtype_in, p.dtype_out, p.alpha, p.beta, p.outer_a, p.outer_b)
    probe_a = torch.empty(max(p.vol_a, 1), dtype=H.torch_dtype(p.dtype_in), device="cuda")
    probe_b = torch.empty(max(p.vol_b, 1), dtype=H.torch_dtype(p.dtype_out), device="cuda")
    for i in range(plan.info()["ncandidates"]):
        plan.select(i)
        try:
            plan.execute_noalloc(probe_a, probe_b)
            torch.cuda.synchronize()
            return plan
        except ttc.TTCError as e:
            assert e.name == "TTC_ERR_INVALID_SIZE", str(e)
    pytest.fail(f"no schedule of {p.tag} fits the static scratch")


@pytest.mark.parametrize("p", CASES, ids=lambda p: p.tag)
def test_noalloc_matches_execute_on_two_calls(p):
    plan = fitting_plan(p)
    A, B0 = H.make_inputs(p, 17, "normal")
    want, want_scale = H.oracle_mirror(p, A, B0)
    dA = H.to_device(A, p.dtype_in)
    # the regular entry point
    dB = H.to_device(B0, p.dtype_out)
    plan.execute(dA, dB)
    ref_scale = None
    if p.dtype_out == "e4m3":
        s = torch.zeros(1, dtype=torch.float32, device="cuda")
        plan.get_fp8_scale(s)
        ref_scale = float(s.cpu().item())
    torch.cuda.synchronize()
    ref = H.to_host(dB, p.dtype_out)
    # the allocation-free entry point, twice in a row
    for call in range(2):
        dB2 = H.to_device(B0, p.dtype_out)
        s2 = torch.full((1,), float("nan"), dtype=torch.float32, device="cuda")
        plan.execute_noalloc(dA, dB2, s2 if p.dtype_out == "e4m3" else None)
        torch.cuda.synchronize()
        got = H.to_host(dB2, p.dtype_out)
        ok, msg = H.compare_bits(got, want, p.dtype_out, nan_as_nan=True)
        assert ok, f"call {call} against the oracle: {msg}"
        ok, msg = H.compare_bits(got, ref, p.dtype_out, nan_as_nan=True)
        assert ok, f"call {call} against ttc_execute: {msg}"
        if p.dtype_out == "e4m3":
            assert float(s2.cpu().item()) == ref_scale == want_scale, f"call {call}: scale"


@pytest.mark.parametrize("p", CASES, ids=lambda p: p.tag)
def test_noalloc_first_call_leaves_free_device_memory_unchanged(p):
    """A fresh plan's first call allocates nothing: the device's free memory
    (cudaMemGetInfo) is the same before and after it.  An earlier plan of the
    same problem has run the same kernels, so that loading their code (which
    the CUDA driver may do on a kernel's first launch) does not show up here."""
    fitting_plan(p)                        # loads the kernels of this schedule
    fresh = fitting_plan(p)
    sel = fresh.info()["candidate"]
    plan = ttc.Plan(p.perm, p.sizes, p.dtype_in, p.dtype_out, p.alpha, p.beta, p.outer_a, p.outer_b)
    plan.select(sel)
    A, B0 = H.make_inputs(p, 23, "normal")
    want, _ = H.oracle_mirror(p, A, B0)
    dA = H.to_device(A, p.dtype_in)
    dB = H.to_device(B0, p.dtype_out)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    plan.execute_noalloc(dA, dB)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, f"free device memory changed by {free0 - free1} bytes"
    ok, msg = H.compare_bits(H.to_host(dB, p.dtype_out), want, p.dtype_out, nan_as_nan=True)
    assert ok, msg


def test_noalloc_two_plans_on_two_streams_ordered_by_an_event():
    """The array is shared: the second stream waits on an event recorded after
    the first plan's call, so the two calls run back to back, and each result
    is that plan's."""
    p1, p2 = CASES[3], CASES[2]                # both upload offset tables
    plan1, plan2 = fitting_plan(p1), fitting_plan(p2)
    A1, B1 = H.make_inputs(p1, 5, "normal")
    A2, B2 = H.make_inputs(p2, 6, "normal")
    w1, _ = H.oracle_mirror(p1, A1, B1)
    w2, _ = H.oracle_mirror(p2, A2, B2)
    dA1, dA2 = H.to_device(A1, p1.dtype_in), H.to_device(A2, p2.dtype_in)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    for _ in range(2):
        o1 = H.to_device(B1, p1.dtype_out)
        o2 = H.to_device(B2, p2.dtype_out)
        torch.cuda.synchronize()
        ev = torch.cuda.Event()
        plan1.execute_noalloc(dA1, o1, stream=s1)
        ev.record(s1)
        s2.wait_event(ev)
        plan2.execute_noalloc(dA2, o2, stream=s2)
        torch.cuda.synchronize()
        ok, msg = H.compare_bits(H.to_host(o1, p1.dtype_out), w1, p1.dtype_out, nan_as_nan=True)
        assert ok, msg
        ok, msg = H.compare_bits(H.to_host(o2, p2.dtype_out), w2, p2.dtype_out, nan_as_nan=True)
        assert ok, msg


def test_noalloc_interleaved_plans_share_the_array():
    """Another plan's call in between leaves nothing behind that changes the result."""
    p1, p2 = CASES[0], CASES[2]
    plan1, plan2 = fitting_plan(p1), fitting_plan(p2)
    A1, B1 = H.make_inputs(p1, 3, "normal")
    A2, B2 = H.make_inputs(p2, 4, "normal")
    dA1, dA2 = H.to_device(A1, p1.dtype_in), H.to_device(A2, p2.dtype_in)
    r1 = H.to_device(B1, p1.dtype_out)
    r2 = H.to_device(B2, p2.dtype_out)
    plan1.execute(dA1, r1)
    plan2.execute(dA2, r2)
    torch.cuda.synchronize()
    for _ in range(2):
        o1 = H.to_device(B1, p1.dtype_out)
        o2 = H.to_device(B2, p2.dtype_out)
        plan1.execute_noalloc(dA1, o1)
        plan2.execute_noalloc(dA2, o2)
        torch.cuda.synchronize()
        assert H.compare_bits(H.to_host(o1, p1.dtype_out), H.to_host(r1, p1.dtype_out), p1.dtype_out, True)[0]
        assert H.compare_bits(H.to_host(o2, p2.dtype_out), H.to_host(r2, p2.dtype_out), p2.dtype_out, True)[0]


def test_noalloc_refuses_schedules_beyond_the_static_scratch():
    # a shape whose candidate list holds tiles with multi-index groups on both
    # sides, i.e. cross-offset tables of several thousand entries
    p = Problem(perm=(1, 0, 3, 2), sizes=(70, 3, 70, 3))
    plan = ttc.Plan(p.perm, p.sizes)
    dA = torch.zeros(p.vol_a, dtype=torch.float32, device="cuda")
    dB = torch.zeros(p.vol_b, dtype=torch.float32, device="cuda")
    refused = 0
    for i in range(plan.info()["ncandidates"]):
        plan.select(i)
        try:
            plan.execute_noalloc(dA, dB)
        except ttc.TTCError as e:
            assert e.name == "TTC_ERR_INVALID_SIZE"
            assert f"the static scratch holds {STATIC_SCRATCH_BYTES}" in str(e)
            refused += 1
            plan.execute(dA, dB)          # the regular entry point still runs it
    torch.cuda.synchronize()
    assert refused >= 1
