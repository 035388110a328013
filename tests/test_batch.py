"""Batches (ttc_batch_*): many problems in one persistent launch, checked
problem by problem against the CPU oracle and against single executions."""
import numpy as np
import pytest

import oracle
from paper_1607_01249_gb300 import build as ttc_build
from paper_1607_01249_gb300 import inputs
from paper_1607_01249_gb300 import ttc
from paper_1607_01249_gb300.inputs import Problem


@pytest.fixture(scope="module", autouse=True)
def built():
    ttc_build.build()
    ttc.lib()


def test_batch_rejects_fp8_and_overlap_on_the_host():
    b = ttc.Batch()
    p8 = ttc.Plan((1, 0), (8, 8), "f32", "e4m3")
    with pytest.raises(ttc.TTCError) as ei:
        b.add(p8, 0x100000, 0x200000)
    assert ei.value.name == "TTC_ERR_UNSUPPORTED_DTYPE"
    p = ttc.Plan((1, 0), (64, 32))
    with pytest.raises(ttc.TTCError) as ei:
        b.add(p, 0x100000, 0x100000 + 1024)
    assert ei.value.name == "TTC_ERR_ALIAS"
    with pytest.raises(ttc.TTCError) as ei:
        b.add(p, 0x100002, 0x200000)
    assert ei.value.name == "TTC_ERR_ALIGN"
    b.add(p, 0x100000, 0x200000)
    b.add(ttc.Plan((1, 0), (0, 5)), 0, 0)          # empty problems are allowed
    info = b.info()
    assert info["problems"] == 2 and info["tiles"] >= 1


def mixed_problems(count, seed):
    g = inputs.rng(seed)
    pairs = [("f32", "f32"), ("bf16", "bf16"), ("f64", "f64"), ("f32", "bf16"), ("f32", "f64"),
             ("f64", "f32"), ("bf16", "f32")]
    out = []
    for i in range(count):
        N = int(g.integers(1, 6))
        perm = tuple(int(x) for x in g.permutation(N))
        n = int(2 ** g.uniform(4, 15))
        sizes = inputs.near_equal_sizes(N, n, g, tol=0.5, min_size=1)
        din, dout = pairs[i % len(pairs)]
        beta = [0.0, 0.5][int(g.integers(2))]
        alpha = [1.0, 1.7][int(g.integers(2))]
        oa = tuple(s + int(g.integers(0, 3)) for s in sizes) if g.random() < 0.3 else None
        if i % 11 == 0:                                    # long runs kept in place: the copy path
            perm, sizes, oa = (0, 2, 1), (3000 + i, 3, 2), None
        out.append(Problem(perm=perm, sizes=sizes, dtype_in=din, dtype_out=dout, alpha=alpha, beta=beta,
                           outer_a=oa))
    return out


@pytest.mark.gpu
def test_batch_matches_oracle_and_single_calls():
    torch = pytest.importorskip("torch")
    from tests import gpu_helpers as H
    probs = mixed_problems(60, 5)
    b = ttc.Batch()
    data = []
    for i, p in enumerate(probs):
        plan = ttc.Plan(p.perm, p.sizes, p.dtype_in, p.dtype_out, p.alpha, p.beta, p.outer_a, p.outer_b)
        A, B0 = H.make_inputs(p, 100 + i, "normal")
        dA, dB = H.to_device(A, p.dtype_in), H.to_device(B0, p.dtype_out)
        b.add(plan, dA, dB)
        data.append((p, plan, A, B0, dA, dB))
    assert b.info()["problems"] == len(probs)
    b.execute()
    torch.cuda.synchronize()
    for p, plan, A, B0, dA, dB in data:
        got = H.to_host(dB, p.dtype_out)
        want, _ = H.oracle_mirror(p, A, B0)
        bitcopy = p.alpha == 1.0 and p.beta == 0.0 and p.dtype_in == p.dtype_out
        ok, msg = H.compare_bits(got, want, p.dtype_out, nan_as_nan=not bitcopy)
        assert ok, (p, msg)
    # same results alone and in the batch
    for p, plan, A, B0, dA, dB in data[:12]:
        single, _ = H.run_gpu(p, A, B0, plan=plan)
        assert H.compare_bits(single, H.to_host(dB, p.dtype_out), p.dtype_out, True)[0]


def test_batch_autotune_argument_checks_on_the_host():
    b = ttc.Batch()
    with pytest.raises(ttc.TTCError) as ei:
        b.autotune(0)
    assert ei.value.name == "TTC_ERR_INVALID_ARG"
    assert b.autotune(4) == 0          # an empty batch has nothing to time


@pytest.mark.gpu
def test_autotuned_batch_matches_oracle_and_leaves_tensors_alone():
    """ttc_batch_autotune times each plan's batch-body schedules on its own
    buffers: the caller's tensors are unchanged by it, and the batch built
    from the chosen schedules (executed and replayed as a graph) still gives
    the oracle's result for every problem."""
    torch = pytest.importorskip("torch")
    from tests import gpu_helpers as H
    probs = [p for p in mixed_problems(40, 21) if p.beta == 0.0]
    b = ttc.Batch()
    data = []
    for i, p in enumerate(probs):
        plan = ttc.Plan(p.perm, p.sizes, p.dtype_in, p.dtype_out, p.alpha, p.beta, p.outer_a, p.outer_b)
        A, B0 = H.make_inputs(p, 700 + i, "normal")
        dA, dB = H.to_device(A, p.dtype_in), H.to_device(B0, p.dtype_out)
        b.add(plan, dA, dB)
        data.append((p, A, B0, dA, dB))
    b.execute()                          # the cost model's schedules first
    torch.cuda.synchronize()
    before = [H.to_host(dB, p.dtype_out).copy() for p, A, B0, dA, dB in data]
    changed = b.autotune(4)
    torch.cuda.synchronize()
    assert 0 <= changed <= len(probs)
    for (p, A, B0, dA, dB), got in zip(data, before):
        assert np.array_equal(H.to_host(dB, p.dtype_out).view(np.uint8), got.view(np.uint8)), p
        assert np.array_equal(H.to_host(dA, p.dtype_in).view(np.uint8), A.view(np.uint8)), p
    for launch in ("execute", "graph_launch"):
        for p, A, B0, dA, dB in data:
            dB.zero_()
        getattr(b, launch)()
        torch.cuda.synchronize()
        for p, A, B0, dA, dB in data:
            want, _ = H.oracle_mirror(p, A, np.zeros_like(B0))
            bitcopy = p.alpha == 1.0 and p.dtype_in == p.dtype_out
            ok, msg = H.compare_bits(H.to_host(dB, p.dtype_out), want, p.dtype_out, nan_as_nan=not bitcopy)
            assert ok, (launch, p, msg)


@pytest.mark.gpu
def test_batch_graph_replay():
    torch = pytest.importorskip("torch")
    from tests import gpu_helpers as H
    probs = [p for p in mixed_problems(24, 9) if p.beta == 0.0]     # replay must not accumulate
    b = ttc.Batch()
    data = []
    for i, p in enumerate(probs):
        plan = ttc.Plan(p.perm, p.sizes, p.dtype_in, p.dtype_out, p.alpha, p.beta, p.outer_a, p.outer_b)
        A, B0 = H.make_inputs(p, 300 + i, "uniform")
        dA, dB = H.to_device(A, p.dtype_in), H.to_device(B0, p.dtype_out)
        b.add(plan, dA, dB)
        data.append((p, A, B0, dB))
    for rep in range(3):
        for p, A, B0, dB in data:
            dB.zero_()
        b.graph_launch()
        torch.cuda.synchronize()
        for p, A, B0, dB in data:
            want, _ = H.oracle_mirror(p, A, np.zeros_like(B0))
            ok, msg = H.compare_bits(H.to_host(dB, p.dtype_out), want, p.dtype_out, True)
            assert ok, (rep, p, msg)


@pytest.mark.gpu
@pytest.mark.parametrize("threshold", [1 << 17, 0])
def test_batch_with_direct_problems_matches_oracle(threshold):
    """Problems at or above the direct threshold run as their own kernels on
    the batch's side stream, beside the persistent kernel that takes the rest;
    both ways, and through a graph, every problem matches the oracle."""
    torch = pytest.importorskip("torch")
    from tests import gpu_helpers as H
    g = inputs.rng(17)
    probs = []
    for i in range(14):
        N = int(g.integers(2, 5))
        n = int(2 ** (g.uniform(17.2, 18.5) if i % 3 == 0 else g.uniform(8, 14)))
        sizes = inputs.near_equal_sizes(N, n, g, tol=0.3, min_size=1)
        perm = inputs.random_perm(N, g)
        dt = ("f32", "bf16", "f64")[i % 3]
        probs.append(Problem(perm=perm, sizes=sizes, dtype_in=dt, dtype_out=dt, alpha=1.5, beta=0.0))
    assert sum(p.n >= (1 << 17) for p in probs) >= 3
    b = ttc.Batch().set_direct_threshold(threshold)
    data = []
    for i, p in enumerate(probs):
        plan = ttc.Plan(p.perm, p.sizes, p.dtype_in, p.dtype_out, p.alpha, p.beta)
        A, B0 = H.make_inputs(p, 500 + i, "normal")
        dA, dB = H.to_device(A, p.dtype_in), H.to_device(B0, p.dtype_out)
        b.add(plan, dA, dB)
        data.append((p, A, B0, dB))
    for launch in (b.execute, b.graph_launch, b.graph_launch):
        for p, A, B0, dB in data:
            dB.zero_()
        launch()
        torch.cuda.synchronize()
        for p, A, B0, dB in data:
            want, _ = H.oracle_mirror(p, A, np.zeros_like(B0))
            ok, msg = H.compare_bits(H.to_host(dB, p.dtype_out), want, p.dtype_out, True)
            assert ok, (threshold, p, msg)
