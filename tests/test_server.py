"""Server (ttc_server_*): requests submitted over time, admitted under a byte
budget, batched into epochs on several streams; each request's result must
equal the oracle's and the result of the same request run alone."""
import time

import numpy as np
import pytest

from paper_1607_01249_gb300 import build as ttc_build
from paper_1607_01249_gb300 import inputs
from paper_1607_01249_gb300 import ttc
from paper_1607_01249_gb300.inputs import Problem


@pytest.fixture(scope="module", autouse=True)
def built():
    ttc_build.build()
    ttc.lib()


@pytest.mark.parametrize("budget,nstreams,small", [(0, 1, 0), (-5, 1, 0), (1 << 20, 0, 0), (1 << 20, 17, 0),
                                                   (1 << 20, 2, -1)])
def test_server_rejects_bad_configuration_on_the_host(budget, nstreams, small):
    with pytest.raises(ttc.TTCError) as ei:
        ttc.Server(budget, nstreams, small)
    assert ei.value.name == "TTC_ERR_INVALID_ARG"


def serving_mix(count, seed):
    """Small and large requests of every batchable pair plus FP8 and packed
    (outer-size) ones."""
    g = inputs.rng(seed)
    pairs = [("f32", "f32"), ("f64", "f64"), ("bf16", "bf16"), ("f32", "bf16"), ("bf16", "f32"),
             ("f32", "e4m3"), ("f64", "f32")]
    out = []
    for i in range(count):
        N = int(g.integers(2, 7))
        perm = tuple(int(x) for x in g.permutation(N))
        if perm == tuple(range(N)):
            perm = perm[1:] + perm[:1]
        n = int(2 ** g.uniform(8, 21 if i % 5 == 0 else 14))
        sizes = inputs.near_equal_sizes(N, n, g, tol=0.5, min_size=1)
        din, dout = pairs[i % len(pairs)]
        beta = 0.0 if dout == "e4m3" else [0.0, 0.4][int(g.integers(2))]
        alpha = [1.0, 1.7][int(g.integers(2))]
        oa = tuple(s + int(g.integers(0, 4)) for s in sizes) if i % 10 == 3 else None
        out.append(Problem(perm=perm, sizes=sizes, dtype_in=din, dtype_out=dout, alpha=alpha, beta=beta,
                           outer_a=oa))
    return out


def run_server(probs, budget, nstreams, small, seed0, spread_s=0.0, shared_fp8_plan=False):
    import torch
    from tests import gpu_helpers as H
    srv = ttc.Server(budget, nstreams, small)
    data = []
    fp8_plan = {}
    for i, p in enumerate(probs):
        if shared_fp8_plan and p.dtype_out == "e4m3":
            key = (p.perm, p.sizes, p.dtype_in, p.alpha, p.outer_a)
            plan = fp8_plan.setdefault(key, ttc.Plan(p.perm, p.sizes, p.dtype_in, p.dtype_out, p.alpha, p.beta,
                                                     p.outer_a, p.outer_b))
        else:
            plan = ttc.Plan(p.perm, p.sizes, p.dtype_in, p.dtype_out, p.alpha, p.beta, p.outer_a, p.outer_b)
        A, B0 = H.make_inputs(p, seed0 + i, "normal")
        data.append([p, plan, A, B0, H.to_device(A, p.dtype_in), H.to_device(B0, p.dtype_out), None])
    torch.cuda.synchronize()
    for d in data:
        d[6] = srv.submit(d[1], d[4], d[5])
        if spread_s:
            time.sleep(spread_s)
    srv.drain(120_000_000)
    for d in data:
        assert srv.poll(d[6], 0)
    st = srv.stats()
    srv.close()
    return data, st


def check_against_oracle(data):
    from tests import gpu_helpers as H
    for p, plan, A, B0, dA, dB, _ in data:
        got = H.to_host(dB, p.dtype_out)
        want, _ = H.oracle_mirror(p, A, B0)
        bitcopy = p.alpha == 1.0 and p.beta == 0.0 and p.dtype_in == p.dtype_out
        ok, msg = H.compare_bits(got, want, p.dtype_out, nan_as_nan=not bitcopy)
        assert ok, (p, msg)


@pytest.mark.gpu
@pytest.mark.parametrize("nstreams,small", [(4, 4096), (2, 64), (1, 0)])
def test_server_results_match_oracle(nstreams, small):
    probs = serving_mix(48, 21)
    data, st = run_server(probs, 1 << 30, nstreams, small, 500)
    assert st["submitted"] == len(probs) and st["completed"] == len(probs) and st["failed"] == 0
    assert st["peak_inflight_bytes"] <= 1 << 30
    if small == 0:
        assert st["launches"] >= len(probs)
    check_against_oracle(data)


@pytest.mark.gpu
def test_server_same_result_alone_and_in_the_mix():
    from tests import gpu_helpers as H
    probs = serving_mix(30, 33)
    data, _ = run_server(probs, 1 << 30, 3, 4096, 900, spread_s=0.0005)
    for p, plan, A, B0, dA, dB, _ in data:
        single, _ = H.run_gpu(p, A, B0)
        ok, msg = H.compare_bits(single, H.to_host(dB, p.dtype_out), p.dtype_out, True)
        assert ok, (p, msg)


@pytest.mark.gpu
def test_server_budget_limits_what_is_in_flight():
    probs = [p for p in serving_mix(40, 44) if p.dtype_out != "e4m3"]
    spans = [p.vol_a * ttc.DTYPE_BYTES[p.dtype_in] + p.vol_b * ttc.DTYPE_BYTES[p.dtype_out] for p in probs]
    budget = max(spans)             # admits little more than one large request at a time
    data, st = run_server(probs, budget, 4, 4096, 1300)
    assert st["peak_inflight_bytes"] <= budget
    assert st["completed"] == len(probs)
    check_against_oracle(data)


@pytest.mark.gpu
def test_server_rejects_requests_over_budget_and_bad_tickets():
    import torch
    p = ttc.Plan((1, 0), (256, 256))
    A = torch.zeros(256 * 256, dtype=torch.float32, device="cuda")
    B = torch.zeros(256 * 256, dtype=torch.float32, device="cuda")
    srv = ttc.Server(256 * 256 * 8 - 1, 2, 1024)
    with pytest.raises(ttc.TTCError) as ei:
        srv.submit(p, A, B)
    assert ei.value.name == "TTC_ERR_BUDGET"
    with pytest.raises(ttc.TTCError) as ei:
        srv.submit(p, A, A)
    assert ei.value.name in ("TTC_ERR_ALIAS", "TTC_ERR_BUDGET")
    with pytest.raises(ttc.TTCError) as ei:
        srv.poll(0)
    assert ei.value.name == "TTC_ERR_INVALID_ARG"
    srv.close()
    srv = ttc.Server(1 << 22, 2, 1024)
    with pytest.raises(ttc.TTCError) as ei:
        srv.submit(p, A, A)
    assert ei.value.name == "TTC_ERR_ALIAS"
    t = srv.submit(p, A, B)
    srv.drain(10_000_000)
    assert srv.poll(t, 0)
    e = srv.submit(ttc.Plan((1, 0), (0, 7)), 0, 0)            # empty request completes at once
    assert srv.poll(e, 0)
    srv.close()


@pytest.mark.gpu
def test_server_fp8_requests_of_one_plan_run_in_turn():
    probs = [Problem(perm=(2, 0, 1), sizes=(40, 33, 70), dtype_in="f32", dtype_out="e4m3", alpha=1.3)] * 6
    data, st = run_server(probs, 1 << 30, 4, 4096, 1700, shared_fp8_plan=True)
    assert st["completed"] == 6
    check_against_oracle(data)


@pytest.mark.gpu
def test_server_watchdog_gives_up_an_epoch_and_keeps_serving():
    """Failure detection without a GPU fault: a request whose kernel stays
    busy (bounded, 0.4 s) longer than the watchdog (0.1 s) completes with
    TTC_ERR_TIMEOUT, its stream is retired, the other streams keep serving,
    and the server shuts down without waiting for the given-up stream."""
    import torch
    from tests import gpu_helpers as H
    srv = ttc.Server(1 << 30, 2, 4096)
    probs = [Problem(perm=(1, 0), sizes=(300, 200)), Problem(perm=(2, 0, 1), sizes=(64, 50, 70), alpha=1.5)]

    def serve_all():
        data = []
        for i, p in enumerate(probs):
            plan = ttc.Plan(p.perm, p.sizes, p.dtype_in, p.dtype_out, p.alpha, p.beta)
            A, B0 = H.make_inputs(p, 40 + i)
            dA, dB = H.to_device(A, p.dtype_in), H.to_device(B0, p.dtype_out)
            data.append((p, A, B0, dB, srv.submit(plan, dA, dB)))
        for p, A, B0, dB, t in data:
            assert srv.poll(t, 5_000_000)
            torch.cuda.synchronize()
            want, _ = H.oracle_mirror(p, A, B0)
            assert H.compare_bits(H.to_host(dB, p.dtype_out), want, p.dtype_out, True)[0]

    # once under the default watchdog: the first launches of the serving
    # kernels (whose code the driver may load then) are not what the short
    # watchdog below is about
    serve_all()
    srv.set_watchdog(0.1)
    t_slow = srv.submit_delay(400_000)
    with pytest.raises(ttc.TTCError) as ei:
        srv.poll(t_slow, 3_000_000)
    assert ei.value.name == "TTC_ERR_TIMEOUT"
    serve_all()
    st = srv.stats()
    assert st["failed"] == 1 and st["completed"] == 2 * len(probs)
    t0 = time.time()
    srv.close()
    assert time.time() - t0 < 5.0
    torch.cuda.synchronize()          # the delay kernel has ended on its own
