"""Host-side tests of libttc (no GPU): exports, validation, canonicalisation,
schedule choice, and the checks ttc_execute makes before touching the device."""
import ctypes
import math
import os
import re
import subprocess

import pytest

from paper_1607_01249_gb300 import build as ttc_build
from paper_1607_01249_gb300 import inputs
from paper_1607_01249_gb300 import ttc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden")


@pytest.fixture(scope="module", autouse=True)
def built():
    ttc_build.build()
    ttc.lib()


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "ttc.h")).read() + open(os.path.join(ROOT, "include", "ttc_debug.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(ttc_[a-z0-9_]+)\s*\(", txt)))


def test_exports_every_declared_symbol():
    names = declared_functions()
    assert "ttc_plan" in names and "ttc_execute" in names
    out = subprocess.run(["nm", "-D", "--defined-only", ttc.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(l.split()[-1] for l in out.splitlines() if l.strip())
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert n in ttc.SIGNATURES, f"binding lacks {n}"


def test_status_strings():
    L = ttc.lib()
    for code, name in ttc.STATUS.items():
        assert L.ttc_status_string(code).decode() == name


@pytest.mark.parametrize("perm,sizes,outer_a,outer_b,status", [
    ((0, 0), (2, 3), None, None, "TTC_ERR_INVALID_PERM"),
    ((0, 2), (2, 3), None, None, "TTC_ERR_INVALID_PERM"),
    ((1, 0), (2, -3), None, None, "TTC_ERR_INVALID_SIZE"),
    ((1, 0), (4, 3), (3, 3), None, "TTC_ERR_INVALID_OUTER"),
    ((1, 0), (4, 3), None, (2, 4), "TTC_ERR_INVALID_OUTER"),
    ((1, 0), (1 << 40, 1 << 40), None, None, "TTC_ERR_INVALID_SIZE"),
])
def test_plan_validation(perm, sizes, outer_a, outer_b, status):
    with pytest.raises(ttc.TTCError) as ei:
        ttc.Plan(perm, sizes, outer_a=outer_a, outer_b=outer_b)
    assert ei.value.name == status


def test_plan_validation_ndim_and_dtypes():
    with pytest.raises(ttc.TTCError) as ei:
        ttc.Plan(tuple(range(17)), (1,) * 17)
    assert ei.value.name == "TTC_ERR_INVALID_PERM"
    for din, dout in [("f64", "bf16"), ("f64", "e4m3"), ("e4m3", "f32"), ("bf16", "f64")]:
        with pytest.raises(ttc.TTCError) as ei:
            ttc.Plan((1, 0), (4, 4), din, dout)
        assert ei.value.name == "TTC_ERR_UNSUPPORTED_DTYPE"
    with pytest.raises(ttc.TTCError) as ei:
        ttc.Plan((1, 0), (4, 4), "f32", "e4m3", beta=0.5)
    assert ei.value.name == "TTC_ERR_UNSUPPORTED_DTYPE"
    for din, dout in [("f32", "f32"), ("f32", "f64"), ("f32", "bf16"), ("f32", "e4m3"), ("f64", "f64"),
                      ("f64", "f32"), ("bf16", "bf16"), ("bf16", "f32"), ("bf16", "e4m3"), ("c64", "c64"),
                      ("c128", "c128"), ("c64", "c128"), ("c128", "c64")]:
        ttc.Plan((1, 0), (4, 4), din, dout)


def test_complex_plan_validation():
    """Complex types pair only with complex types; complex scalars need
    complex tensors; every part of alpha and beta must be finite."""
    for din, dout in [("c64", "f32"), ("f64", "c128"), ("c64", "bf16"), ("c128", "e4m3"), ("bf16", "c64")]:
        with pytest.raises(ttc.TTCError) as ei:
            ttc.Plan((1, 0), (4, 4), din, dout)
        assert ei.value.name == "TTC_ERR_UNSUPPORTED_DTYPE"
    for din in ("f32", "f64", "bf16"):
        with pytest.raises(ttc.TTCError) as ei:
            ttc.Plan((1, 0), (4, 4), din, din, alpha=1 + 1j)
        assert ei.value.name == "TTC_ERR_UNSUPPORTED_DTYPE"
    with pytest.raises(ttc.TTCError) as ei:
        ttc.Plan((1, 0), (4, 4), "c64", "c64", alpha=complex(1.0, float("inf")))
    assert ei.value.name == "TTC_ERR_INVALID_ARG"
    p = ttc.Plan((2, 0, 1), (5, 6, 7), "c128", "c64", alpha=0.5j, beta=-1j)
    assert p.info()["algorithmic_bytes"] == 210 * (16 + 2 * 8)     # beta != 0: B read and written
    p = ttc.Plan((2, 0, 1), (5, 6, 7), "c64", "c128", alpha=0.5j)
    assert p.info()["algorithmic_bytes"] == 210 * (8 + 16)
    # not batched: the persistent kernel covers the real pairs only
    b = ttc.Batch()
    with pytest.raises(ttc.TTCError) as ei:
        b.add(ttc.Plan((1, 0), (8, 8), "c64", "c64"), 1 << 20, 2 << 20)
    assert ei.value.name == "TTC_ERR_UNSUPPORTED_DTYPE"
    b.close()


def test_complex_schedules_are_sound():
    """Every candidate of complex problems (8- and 16-byte elements, so 8 and
    4 slots per thread): the kernels' index walks and slot tables put every A
    element at its Eq. 1 position in B."""
    g = inputs.rng(32)
    pairs = [("c64", "c64"), ("c128", "c128"), ("c64", "c128"), ("c128", "c64")]
    for trial in range(60):
        N = int(g.integers(1, 6))
        sizes = tuple(int(x) for x in g.integers(1, 12 if N > 3 else 70, size=N))
        perm = tuple(int(x) for x in g.permutation(N))
        oa = tuple(s + int(g.integers(0, 3)) for s in sizes) if g.random() < 0.4 else None
        din, dout = pairs[trial % 4]
        plan = ttc.Plan(perm, sizes, din, dout, alpha=1.5 - 0.5j, beta=(0.5j if trial % 3 else 0.0), outer_a=oa)
        _verify_all(plan, (perm, sizes, oa, din, dout))
    for c in inputs.complex_cases(target=1 << 16):
        _verify_all(ttc.Plan(c.perm, c.sizes, c.dtype_in, c.dtype_out, c.alpha, c.beta), (c.tag, c.dtype_in))


def test_merge_examples_from_the_paper():
    rows = [l for l in open(os.path.join(GOLDEN, "merge_examples.txt")).read().splitlines()
            if l.strip() and not l.startswith("#")]
    assert rows
    for row in rows:
        name, perm, sizes, oa, cperm, csizes, cite = [x.strip() for x in row.split("|")]
        p = ttc.Plan([int(x) for x in perm.split(",")], [int(x) for x in sizes.split(",")],
                     outer_a=None if oa == "-" else [int(x) for x in oa.split(",")])
        inf = p.info()
        assert inf["perm"] == [int(x) for x in cperm.split(",")], name
        assert inf["sizes"] == [int(x) for x in csizes.split(",")], name


def test_canonical_form_properties():
    g = inputs.rng(21)
    for _ in range(300):
        N = int(g.integers(1, 7))
        sizes = tuple(int(x) for x in g.integers(1, 5, size=N))
        perm = tuple(int(x) for x in g.permutation(N))
        oa = tuple(s + int(g.integers(0, 2)) for s in sizes) if g.random() < 0.3 else None
        p = ttc.Plan(perm, sizes, outer_a=oa)
        inf = p.info()
        n = 1
        for s in sizes:
            n *= s
        assert inf["n"] == n
        prod = 1
        for s in inf["sizes"]:
            prod *= s
        assert prod == n
        assert sorted(inf["perm"]) == list(range(inf["ndim"]))
        assert all(s > 1 for s in inf["sizes"]) or inf["ndim"] == 1
        # no two neighbours that could still merge
        for k in range(inf["ndim"] - 1):
            posb = inf["perm"].index(k)
            adjacent = posb + 1 < inf["ndim"] and inf["perm"][posb + 1] == k + 1
            dense = (inf["stride_A"][k + 1] == inf["stride_A"][k] * inf["sizes"][k] and
                     inf["stride_B"][k + 1] == inf["stride_B"][k] * inf["sizes"][k])
            assert not (adjacent and dense)
        if inf["perm"][0] == 0:
            assert inf["variant"] in ("copy", "tile", "rowcopy")
        elif inf["variant"] == "tma_tile":
            # the TMA tile: two swapped indices, A's column stride 16-byte aligned
            assert inf["ndim"] == 2 and (inf["stride_A"][1] * 4) % 16 == 0
        else:
            assert inf["variant"] == "tile"


def test_schedule_of_the_workloads():
    p0 = inputs.single_4d()
    inf = ttc.Plan(p0.perm, p0.sizes).info()
    assert inf["variant"] == "tile" and inf["ndim"] == 4
    assert inf["algorithmic_bytes"] == p0.n * 8
    for case in inputs.sweep_cases(perms_per_n=8, dtypes=("f32",), betas=(0.0,)):
        inf = ttc.Plan(case.perm, case.sizes, alpha=case.alpha).info()
        c, a, b = inf["tile"]
        if inf["variant"] == "tile":
            # 16 four-byte elements per thread: 256 threads, or 512 for the
            # packed-lane kernel
            assert c * a * b <= 16 * (inf["packed_threads"] or 256)
        assert inf["ncandidates"] >= 1
    for case in inputs.packing_cases():
        inf = ttc.Plan(case.perm, case.sizes, case.dtype_in, case.dtype_out, outer_a=case.outer_a).info()
        assert inf["n"] == case.n


def test_empty_problem_is_a_noop():
    p = ttc.Plan((1, 0), (0, 5))
    assert p.info()["variant"] == "empty"
    p.execute(0, 0)          # no pointers needed, no device touched


def test_execute_host_checks_before_any_device_work():
    p = ttc.Plan((1, 0), (64, 32))
    with pytest.raises(ttc.TTCError) as ei:
        p.execute(0, 0x10000)
    assert ei.value.name == "TTC_ERR_INVALID_ARG"
    with pytest.raises(ttc.TTCError) as ei:
        p.execute(0x10002, 0x100000)
    assert ei.value.name == "TTC_ERR_ALIGN"
    # overlapping byte ranges (A spans 8 KiB)
    with pytest.raises(ttc.TTCError) as ei:
        p.execute(0x100000, 0x100000 + 4096)
    assert ei.value.name == "TTC_ERR_ALIAS"
    with pytest.raises(ttc.TTCError) as ei:
        p.execute(0x100000 + 4096, 0x100000)
    assert ei.value.name == "TTC_ERR_ALIAS"


def test_fastdiv_matches_integer_division(tmp_path):
    src = tmp_path / "fd.cpp"
    src.write_text(r'''
#include "ttc_internal.h"
#include <cstdio>
#include <cstdlib>
int main() {
  unsigned long long bad = 0, n_checked = 0;
  unsigned ds[] = {1,2,3,5,7,10,20,36,90,406,641,1000,4095,4096,4097,65535,65536,65537,
                   1000003,16777213,16777216,2147483647u};
  unsigned long long x = 88172645463325252ull;
  for (unsigned d : ds) {
    ttc::FastDiv f = ttc::make_fastdiv(d);
    for (int i = 0; i < 200000; ++i) {
      x ^= x << 13; x ^= x >> 7; x ^= x << 17;
      unsigned n = (unsigned)(x & 0x7fffffffu);
      if (i < 1000) n = i;
      if (i >= 1000 && i < 2000) n = 0x7fffffffu - (i - 1000);
      if (ttc::fast_div(n, f) != n / d) ++bad;
      ++n_checked;
    }
  }
  for (unsigned d = 1; d < 5000; ++d) {
    ttc::FastDiv f = ttc::make_fastdiv(d);
    for (unsigned n = 0; n < 20000; n += 7) { if (ttc::fast_div(n, f) != n / d) ++bad; ++n_checked; }
    for (unsigned n = 0x7fffffffu - 20000; n < 0x7fffffffu; n += 13) { if (ttc::fast_div(n, f) != n / d) ++bad; ++n_checked; }
  }
  printf("%llu %llu\n", bad, n_checked);
  return bad != 0;
}
''')
    exe = tmp_path / "fd"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_1607_01249_gb300", "csrc"),
                           str(src), "-o", str(exe)])
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout


def test_integer_float_conversions_match_ieee_casts(tmp_path):
    """The kernels' binary32 <-> binary64 conversions and binary64 product
    (integer operations, no FP64 instruction) against the host's IEEE
    arithmetic: widening on every one of the 2^32 binary32 values, narrowing
    on exponents across and beyond the binary32 range, exact ties and rounding
    carries, and arbitrary bit patterns (NaN only has to stay NaN); the
    product on random operands of every exponent for several constants."""
    src = tmp_path / "conv.cpp"
    src.write_text(r'''
#include "fpint.h"
#include <cmath>
#include <cstdio>
using namespace ttc;
int main() {
  unsigned long long bad = 0, n = 0;
  for (unsigned long long u = 0; u < (1ull << 32); ++u) {
    const float f = fp_float((uint32_t)u);
    const double a = widen_f32(f), b = (double)f;
    ++n;
    if (std::isnan(b) ? !std::isnan(a) : fp_bits(a) != fp_bits(b)) ++bad;
  }
  unsigned long long x = 88172645463325252ull;
  auto rnd = [&]() { x ^= x << 13; x ^= x >> 7; x ^= x << 17; return x; };
  auto check = [&](unsigned long long bits) {
    const double d = fp_double((uint32_t)(bits >> 32), (uint32_t)bits);
    const float a = narrow_f64_rn(d), b = (float)d;
    ++n;
    if (std::isnan(b) ? !std::isnan(a) : fp_bits(a) != fp_bits(b)) ++bad;
  };
  for (int i = 0; i < 20000000; ++i) {
    const unsigned long long r = rnd();
    const unsigned long long bits = (r & (1ull << 63)) | ((850 + (r >> 20) % 330) << 52) | (rnd() & 0xfffffffffffffull);
    check(bits);
    check((bits & ~0x1fffffffull) | 0x10000000ull);
    check(bits | 0x1fffffffull);
  }
  for (unsigned long long e = 0; e < 2048; ++e)
    for (unsigned long long k = 0; k < 53; ++k) {
      const unsigned long long frac = ((1ull << k) - 1) << (52 - k);
      check((e << 52) | frac);
      check((1ull << 63) | (e << 52) | frac);
      check((e << 52) | (1ull << 28) | ((k & 1) << 29));
    }
  for (int i = 0; i < 5000000; ++i) check(rnd());
  // the integer product fl64(c * a): wherever it claims a result, the host's
  // multiplication gives the same bits
  const double cs[] = {1.7, 0.4, -1.7, 1.0, 0.5, 3.141592653589793, 1e-300, 1e300, 0.1, 1.9999999999999998};
  for (double c : cs) {
    const DMulConst k = make_dmul_const(c);
    for (int i = 0; i < 3000000; ++i) {
      const unsigned long long r = rnd();
      const unsigned long long e = (i & 3) ? 1003 + (r >> 20) % 40 : (r >> 20) % 2048;
      unsigned long long bits = (r & (1ull << 63)) | (e << 52) | (rnd() & 0xfffffffffffffull);
      if (i % 5 == 1) bits &= ~0xffffffffull;
      const double a = fp_double((uint32_t)(bits >> 32), (uint32_t)bits);
      double got;
      ++n;
      if (dmul_normal(k, a, &got) && fp_bits(got) != fp_bits(c * a)) ++bad;
    }
  }
  printf("%llu %llu\n", bad, n);
  return bad != 0;
}
''')
    exe = tmp_path / "conv"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_1607_01249_gb300", "csrc"),
                           str(src), "-o", str(exe)])
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout


def _verify_all(plan, label):
    for i in range(plan.info()["ncandidates"]):
        msg = plan.verify_schedule(i)
        assert msg == "", f"{label} candidate {i}: {msg}"
    for j in range(4):                        # the batched body's schedules (default and autotuned)
        msg = plan.verify_schedule(-1 - j)
        if msg == "no such batch candidate":
            break
        assert msg == "", f"{label} batch schedule {j}: {msg}"


def test_schedules_are_sound_on_random_problems():
    """Every candidate schedule of many random problems: the kernels' own index
    walks stay in bounds and put every A element at its Eq. 1 position in B."""
    g = inputs.rng(31)
    for trial in range(150):
        N = int(g.integers(1, 7))
        sizes = tuple(int(x) for x in g.integers(1, 12 if N > 3 else 90, size=N))
        perm = tuple(int(x) for x in g.permutation(N))
        oa = tuple(s + int(g.integers(0, 3)) for s in sizes) if g.random() < 0.4 else None
        sb = tuple(sizes[q] for q in perm)
        ob = tuple(s + int(g.integers(0, 3)) for s in sb) if g.random() < 0.3 else None
        din, dout = [("f32", "f32"), ("f64", "f64"), ("bf16", "bf16"), ("f32", "e4m3"), ("f32", "bf16")][trial % 5]
        plan = ttc.Plan(perm, sizes, din, dout, outer_a=oa, outer_b=ob)
        _verify_all(plan, (perm, sizes, oa, ob, din, dout))


def test_schedules_are_sound_on_the_workloads():
    p = inputs.single_4d()
    _verify_all(ttc.Plan(p.perm, p.sizes), "single4d")
    for c in inputs.packing_cases():
        _verify_all(ttc.Plan(c.perm, c.sizes, c.dtype_in, c.dtype_out, outer_a=c.outer_a), c.tag)
    # the 2D..6D sweep shapes at a reduced size (same index structure)
    g = inputs.rng(5)
    for N in (2, 3, 4, 5, 6):
        for perm in inputs.sweep_perms(N, g, 8):
            sizes = inputs.near_equal_sizes(N, 1 << 17, g, tol=0.05)
            _verify_all(ttc.Plan(perm, sizes, "f32", "f32", 1.7, 0.4), (perm, sizes))


def test_tune_cache_file_round_trip(tmp_path):
    """The autotune cache is a text file of key<TAB>schedule lines: loading a
    file and saving the cache keeps every entry."""
    src = tmp_path / "in.txt"
    entries = {"GB300-test:0>0:b0:N2:100/1/50/1:50/100/1/0": "tile c=0 ga=[0]/32 gb=[1]/64 j=1,2 order=[1,0]",
               "GB300-test:1>1:b1:N3:7/1/1/0:5/7/35/2:3/35/5/1": "copy chunk=7 vec=1"}
    src.write_text("".join(f"{k}\t{v}\n" for k, v in entries.items()) + "malformed line without a tab\n")
    ttc.tune_cache_load(str(src))
    out = tmp_path / "out.txt"
    ttc.tune_cache_save(str(out))
    got = dict(line.split("\t", 1) for line in out.read_text().splitlines())
    for k, v in entries.items():
        assert got[k] == v
    with pytest.raises(ttc.TTCError) as ei:
        ttc.tune_cache_load(str(tmp_path / "missing.txt"))
    assert ei.value.name == "TTC_ERR_INVALID_ARG"


def test_contraction_plan_validation_and_layouts():
    """TTGT planning on the host: label rules, extents, dtypes, and which
    tensors need a transpose for each layout."""
    C = ttc.Contraction
    bad = [
        (((0, 1), (4, 5), (1, 2), (5, 6), (0, 3), (4, 6)), "TTC_ERR_INVALID_PERM"),     # label 3 only in C
        (((0, 1), (4, 5), (1, 2), (5, 6), (0, 2, 1), (4, 6, 5)), "TTC_ERR_INVALID_PERM"),  # batched label
        (((0, 1, 7), (4, 5, 2), (1, 2), (5, 6), (0, 2), (4, 6)), "TTC_ERR_INVALID_PERM"),  # label 7 in A only
        (((0, 1), (4, 5), (1, 2), (6, 6), (0, 2), (4, 6)), "TTC_ERR_INVALID_SIZE"),      # extent mismatch
        (((0, 0), (4, 4), (0, 2), (4, 6), (2,), (6,)), "TTC_ERR_INVALID_PERM"),         # repeated label
    ]
    for (ma, sa, mb, sb, mc, sc), status in bad:
        with pytest.raises(ttc.TTCError) as ei:
            C(ma, sa, mb, sb, mc, sc)
        assert ei.value.name == status, (ma, mb, mc)
    for dt, gd in [("f64", "f32"), ("f32", "f64"), ("bf16", "bf16"), ("c64", "c64"), ("f64", "bf16")]:
        with pytest.raises(ttc.TTCError) as ei:
            C((0, 1), (4, 5), (1, 2), (5, 6), (0, 2), (4, 6), dt, gd)
        assert ei.value.name == "TTC_ERR_UNSUPPORTED_DTYPE"
    # matrix layouts need no transpose in either orientation; a permuted C does
    assert C((0, 1), (4, 5), (1, 2), (5, 6), (0, 2), (4, 6)).info() == {
        "m": 4, "n": 6, "k": 5, "permuted": {"A": False, "B": False, "C": False}}
    assert C((1, 0), (5, 4), (2, 1), (6, 5), (2, 0), (6, 4)).info()["permuted"] == {"A": False, "B": False,
                                                                                  "C": False}
    # C = [free B, free A]: the GEMM computes C's transpose directly
    inf = C((0, 3, 1, 4), (3, 2, 4, 5), (4, 2, 3), (5, 6, 2), (2, 1, 0), (6, 4, 3)).info()
    assert (inf["m"], inf["n"], inf["k"]) == (12, 6, 10)
    assert inf["permuted"] == {"A": True, "B": True, "C": False}
    # free labels interleaved in C: the product goes through a workspace and a transpose
    inf = C((0, 3, 1, 4), (3, 2, 4, 5), (4, 2, 3), (5, 6, 2), (1, 2, 0), (4, 6, 3)).info()
    assert inf["permuted"]["C"]
    # the BF16 GEMM path always packs (downcasts) both operands
    assert C((0, 1), (4, 5), (1, 2), (5, 6), (0, 2), (4, 6), "f32", "bf16").info()["permuted"] == {
        "A": True, "B": True, "C": False}
    # BF16 plans of every layout kind, including an outer product (no
    # contracted label: a unit contracted index stands in), an empty
    # contracted extent and an empty free extent, are made on the host
    for ma, sa, mb, sb, mc, sc in [((0, 1), (4, 6), (2, 3), (5, 7), (3, 0, 2, 1), (7, 4, 5, 6)),
                                   ((5, 1, 0, 6), (3, 4, 5, 6), (6, 3, 1, 5), (6, 7, 4, 3), (3, 0), (7, 5)),
                                   ((0, 1), (5, 0), (1, 2), (0, 6), (2, 0), (6, 5)),
                                   ((0, 1), (0, 4), (1, 2), (4, 3), (0, 2), (0, 3))]:
        inf = C(ma, sa, mb, sb, mc, sc, "f32", "bf16").info()
        assert inf["m"] * inf["n"] == math.prod(sc)


def test_packed_gemm_plan_on_the_host():
    """ttc_packed_gemm_plan validates and splits the packed panel on the host
    (no device work): M is the product of the first rank_m packed indices, K
    of the rest."""
    g = ttc.PackedGemm((0, 2, 1, 3), (20, 8, 13, 9), 2, 96)
    assert g.info() == {"m": 20 * 13, "n": 96, "k": 8 * 9}
    g = ttc.PackedGemm((0, 1), (4096, 2048), 1, 4096, outer_a=(8192, 8192))
    assert g.info() == {"m": 4096, "n": 4096, "k": 2048}
    for args, status in [(((0, 1), (64, 60), 1, 64), "TTC_ERR_INVALID_SIZE"),      # K not a multiple of 8
                         (((0, 1), (64, 64), 0, 64), "TTC_ERR_INVALID_ARG"),       # rank_m must split
                         (((0, 1), (64, 64), 2, 64), "TTC_ERR_INVALID_ARG"),
                         (((0, 0), (64, 64), 1, 64), "TTC_ERR_INVALID_PERM"),
                         (((0, 1), (64, 64), 1, 0), "TTC_ERR_INVALID_SIZE"),       # n >= 1
                         (((0, 1), (0, 64), 1, 64), "TTC_ERR_INVALID_SIZE")]:
        with pytest.raises(ttc.TTCError) as ei:
            ttc.PackedGemm(*args)
        assert ei.value.name == status, args
    with pytest.raises(ttc.TTCError) as ei:
        ttc.PackedGemm((0, 1), (64, 64), 1, 64, outer_a=(32, 64))
    assert ei.value.name == "TTC_ERR_INVALID_OUTER"
    # execute checks come before any device work
    g = ttc.PackedGemm((0, 1), (64, 64), 1, 64)
    with pytest.raises(ttc.TTCError) as ei:
        g.execute(0x100000, 0x200008, 0x300000)     # B not 16-byte aligned
    assert ei.value.name == "TTC_ERR_ALIGN"
    with pytest.raises(ttc.TTCError) as ei:
        g.execute(0x100000, 0x200000, 0x100000 + 64)  # C inside A
    assert ei.value.name == "TTC_ERR_ALIAS"


def test_contraction_planner_decisions_on_random_layouts():
    """Random contractions (host only): the GEMM extents are the products of
    the free and contracted extents, and an operand is permuted exactly when
    it is not already a matrix in either orientation ([free, contracted] or
    [contracted, free]); C is permuted exactly when it is neither [free A,
    free B] nor [free B, free A] in C's own label order."""
    g = inputs.rng(77)
    for trial in range(200):
        labels = list(range(int(g.integers(2, 7))))
        roles = {}
        for lab in labels:
            roles[lab] = ["k", "a", "b"][int(g.integers(0, 3))]
        ka = [lab for lab in labels if roles[lab] in "ka"]
        kb = [lab for lab in labels if roles[lab] in "kb"]
        kc = [lab for lab in labels if roles[lab] in "ab"]
        if not ka or not kb or not kc:
            continue
        ma = tuple(int(x) for x in g.permutation(ka))
        mb = tuple(int(x) for x in g.permutation(kb))
        mc = tuple(int(x) for x in g.permutation(kc))
        ext = {lab: int(g.integers(1, 6)) for lab in labels}
        c = ttc.Contraction(ma, [ext[m] for m in ma], mb, [ext[m] for m in mb], mc, [ext[m] for m in mc])
        inf = c.info()
        contracted = [m for m in ma if roles[m] == "k"]
        fa_c = [m for m in mc if roles[m] == "a"]
        fb_c = [m for m in mc if roles[m] == "b"]
        prod = lambda ls: math.prod(ext[m] for m in ls)
        assert (inf["m"], inf["n"], inf["k"]) == (prod(fa_c), prod(fb_c), prod(contracted)), (ma, mb, mc)
        c_direct = list(mc) in (fa_c + fb_c, fb_c + fa_c)
        assert inf["permuted"]["C"] == (not c_direct), (ma, mb, mc)
        # the free indices of an operand follow C's order when C is a GEMM
        # output layout, else the operand's own order
        fa = fa_c if c_direct else [m for m in ma if roles[m] == "a"]
        fb = fb_c if c_direct else [m for m in mb if roles[m] == "b"]
        a_matrix = list(ma) in (fa + contracted, contracted + fa)
        b_matrix = list(mb) in (contracted + fb, fb + contracted)
        assert inf["permuted"]["A"] == (not a_matrix), (ma, mb, mc)
        assert inf["permuted"]["B"] == (not b_matrix), (ma, mb, mc)
