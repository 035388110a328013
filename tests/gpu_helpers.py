"""Test infrastructure: run a problem through libttc on the GPU and compare it
with the CPU oracle element by element (bit-exact against the oracle's
rounding sequence, and within the stated tolerance of the exact value)."""
from __future__ import annotations

import math

import numpy as np

import oracle
from paper_1607_01249_gb300 import inputs
from paper_1607_01249_gb300 import ttc

ODT = {"f32": oracle.F32, "f64": oracle.F64, "bf16": oracle.BF16, "e4m3": oracle.E4M3, "c64": oracle.C64,
       "c128": oracle.C128}
COMPLEX = ("c64", "c128")
PART = {"c64": "f32", "c128": "f64"}       # the type of one part of a complex element


def torch_dtype(dt):
    import torch
    return {"f32": torch.float32, "f64": torch.float64, "bf16": torch.int16, "e4m3": torch.uint8}[dt]


def to_device(x: np.ndarray, dt: str):
    import torch
    if dt == "bf16":
        x = x.view(np.int16)
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def to_host(t, dt: str) -> np.ndarray:
    x = t.cpu().numpy()
    if dt == "bf16":
        x = x.view(np.uint16)
    return x


def make_inputs(p: inputs.Problem, seed: int, dist="uniform", b_fill=None):
    A = inputs.tensor_for(p.dtype_in, p.vol_a, seed, dist)
    if b_fill is None:
        B0 = inputs.tensor_for(p.dtype_out, p.vol_b, seed + 1000, dist)
    else:
        B0 = np.full(p.vol_b, b_fill, dtype=inputs.STORAGE[p.dtype_out])
    return A, B0


def run_gpu(p: inputs.Problem, A: np.ndarray, B0: np.ndarray, plan=None, stream=None, scale_dev=None):
    import torch
    plan = plan or ttc.Plan(p.perm, p.sizes, p.dtype_in, p.dtype_out, p.alpha, p.beta, p.outer_a, p.outer_b)
    dA = to_device(A, p.dtype_in)
    dB = to_device(B0, p.dtype_out)
    if scale_dev is not None:
        plan.set_fp8_scale(scale_dev)
    plan.execute(dA, dB, stream)
    scale = None
    if p.dtype_out == "e4m3":
        s = torch.zeros(1, dtype=torch.float32, device="cuda")
        plan.get_fp8_scale(s, stream)
        scale = float(s.cpu().item())
    torch.cuda.synchronize()
    return to_host(dB, p.dtype_out), scale


def oracle_mirror(p: inputs.Problem, A, B0, scale=None):
    Bm = B0.copy()
    if p.dtype_in in COMPLEX:
        oracle.permute_complex(p.perm, p.sizes, A, Bm, p.alpha, p.beta, ODT[p.dtype_in], ODT[p.dtype_out],
                               p.outer_a, p.outer_b)
        return Bm, None
    if p.dtype_out == "e4m3" and scale is None:
        scale, _ = oracle.fp8_scale(p.sizes, A, p.alpha, ODT[p.dtype_in], p.outer_a)
    oracle.permute(p.perm, p.sizes, A, Bm, p.alpha, p.beta, ODT[p.dtype_in], ODT[p.dtype_out],
                   p.outer_a, p.outer_b, fp8_scale=scale if scale is not None else 1.0)
    return Bm, scale


def as_float(x: np.ndarray, dt: str) -> np.ndarray:
    if dt == "bf16":
        return (x.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    if dt == "e4m3":
        return oracle.e4m3_to_f32(x).astype(np.float64)
    return x.astype(np.float64)


def compare_bits(got: np.ndarray, want: np.ndarray, dt: str, nan_as_nan: bool):
    """Bitwise equality; with nan_as_nan, NaN compares equal to any NaN.
    Complex elements compare part by part."""
    if got.dtype != want.dtype or got.shape != want.shape:
        return False, "dtype/shape"
    if dt in COMPLEX:
        pt = np.float32 if dt == "c64" else np.float64
        return compare_bits(got.view(pt), want.view(pt), PART[dt], nan_as_nan)
    if not nan_as_nan:
        eq = got.view(np.uint8).reshape(got.size, -1) == want.view(np.uint8).reshape(want.size, -1)
        bad = np.flatnonzero(~eq.all(axis=1))
    else:
        gf, wf = as_float(got, dt), as_float(want, dt)
        gn, wn = np.isnan(gf), np.isnan(wf)
        ub = {1: np.uint8, 2: np.uint16, 4: np.uint32, 8: np.uint64}[got.dtype.itemsize]
        same = (got.view(ub) == want.view(ub)) | (gn & wn)
        bad = np.flatnonzero(~same)
    if bad.size:
        i = int(bad[0])
        return False, f"{bad.size} mismatches, first at {i}: got {got[i]!r} want {want[i]!r}"
    return True, ""


def tolerance_check(p: inputs.Problem, A, B0, got: np.ndarray):
    """Primary tolerance against the exact value (readings of the precision):
    FP32 data: 2 FP32 ulps at the scale max(|alpha a|, |beta b|, |r|);
    FP64 data: 1e-15 relative at that scale; BF16 output: 1 BF16 ulp."""
    if p.dtype_out == "e4m3":
        return True, ""
    if p.dtype_in in COMPLEX:
        return complex_tolerance_check(p, A, B0, got)
    R, S = oracle.permute_exact(p.perm, p.sizes, A, B0.copy(), p.alpha, p.beta, ODT[p.dtype_in],
                                ODT[p.dtype_out], p.outer_a, p.outer_b)
    mask = ~np.isnan(S)
    g = as_float(got, p.dtype_out)[mask]
    r, s = R[mask], S[mask]
    fin = np.isfinite(r) & np.isfinite(s)
    if not np.all(np.isnan(g[~fin]) == np.isnan(r[~fin])):
        return False, "non-finite mismatch"
    g, r, s = g[fin], r[fin], s[fin]
    err = np.abs(g - r)
    with np.errstate(divide="ignore"):
        e = np.floor(np.log2(np.where(s > 0, s, 1.0)))
    if p.dtype_out == "bf16":
        tol = 2.0 ** (e - 7)
    elif "f64" in (p.dtype_in, p.dtype_out) and p.dtype_out == "f64":
        tol = 1e-15 * s
    else:
        tol = 2.0 * 2.0 ** (e - 23)
    tol = np.where(s > 0, tol, 0.0)
    # smallest subnormal spacing of the output type
    tiny = {"f32": 2.0 ** -149, "f64": 2.0 ** -1074, "bf16": 2.0 ** -133}[p.dtype_out]
    bad = err > np.maximum(tol, tiny)
    if np.any(bad):
        i = int(np.flatnonzero(bad)[0])
        return False, f"{int(bad.sum())} beyond tolerance; first err {err[i]} tol {tol[i]}"
    return True, ""


def complex_tolerance_check(p: inputs.Problem, A, B0, got: np.ndarray):
    """Complex data: each part within the error bound of its rounding
    sequence, 4 roundings in the compute type at the part's scale (the sum of
    the absolute values of its products) plus one rounding to B's type."""
    R, S = oracle.permute_complex_exact(p.perm, p.sizes, A, B0.copy(), p.alpha, p.beta, ODT[p.dtype_in],
                                        ODT[p.dtype_out], p.outer_a, p.outer_b)
    mask = ~np.isnan(S[:, 0])
    eps_c = 2.0 ** -53 if "c128" in (p.dtype_in, p.dtype_out) else 2.0 ** -24
    eps_o = 2.0 ** -24 if p.dtype_out == "c64" else 2.0 ** -53
    tiny = 2.0 ** -149 if p.dtype_out == "c64" else 2.0 ** -1074
    g = got.astype(np.complex128)[mask]
    for k, (gp, rp) in enumerate(((g.real, R.real[mask]), (g.imag, R.imag[mask]))):
        err = np.abs(gp - rp)
        tol = np.maximum(4 * eps_c * S[mask, k] + eps_o * np.abs(rp), tiny)
        bad = err > tol
        if np.any(bad):
            i = int(np.flatnonzero(bad)[0])
            return False, f"{int(bad.sum())} parts beyond tolerance; first err {err[i]} tol {tol[i]}"
    return True, ""


def fp8_error_report(p: inputs.Problem, A, got: np.ndarray, scale: float) -> dict:
    """Error of the dequantised FP8 result against the exact alpha*a."""
    dt_o = "f64" if p.dtype_in == "f32" else "f32"
    R, S = oracle.permute_exact(p.perm, p.sizes, A, np.zeros(p.vol_b, inputs.STORAGE[dt_o]), p.alpha, 0.0,
                                ODT[p.dtype_in], ODT[dt_o], p.outer_a, None)
    deq = as_float(got, "e4m3") * scale
    m = ~np.isnan(R)
    err = np.abs(deq[m] - R[m])
    ref = np.abs(R[m])
    rel = err / np.where(ref > 0, ref, 1.0)
    return {"max_abs": float(err.max(initial=0)), "max_rel": float(rel.max(initial=0)),
            "rms": float(math.sqrt(np.mean(err ** 2))) if err.size else 0.0,
            "bound_ok": bool(np.all(err <= 2.0 ** -4 * ref + scale * 2.0 ** -10 + 1e-30))}


def full_check(p: inputs.Problem, seed=0, dist="uniform", b_fill=None, plan=None):
    A, B0 = make_inputs(p, seed, dist, b_fill)
    got, scale = run_gpu(p, A, B0, plan=plan)
    want, oscale = oracle_mirror(p, A, B0)
    if p.dtype_out == "e4m3":
        assert scale == oscale, (scale, oscale)
    bitcopy = p.alpha == 1.0 and p.beta == 0.0 and p.dtype_in == p.dtype_out
    ok, msg = compare_bits(got, want, p.dtype_out, nan_as_nan=not bitcopy)
    assert ok, f"{p}: mirror {msg}"
    ok, msg = tolerance_check(p, A, B0, got)
    assert ok, f"{p}: tolerance {msg}"
    return A, B0, got, scale
