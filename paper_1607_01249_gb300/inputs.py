"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no arithmetic of the permute-scale-add itself: it only
draws problem descriptions (permutations, sizes, outer sizes, dtypes, scalars)
and random tensor contents from fixed seeds, so that the CUDA path and the CPU
oracle can be fed the same inputs.

Workloads (the paper's 57-case, 2D-6D, 200 MB-per-tensor benchmark of section 3
is not available, so these synthetic families stand in for it):

* ``single_4d``   -- one 4D FP32 transpose, sizes (32,40,24,36), perm (2,0,3,1).
* ``sweep_cases`` -- N = 2..6, 8 seeded random non-identity perms per N,
  near-equal random sizes with 2^26 elements (+-1%), FP32 and FP64,
  alpha = 1.7, beta in {0, 0.4}.
* ``packing_cases`` -- the GEMM packing use of section 2.1 (Figs. 2-3): a
  4096x2048 sub-block of an 8192x8192 column-major matrix viewed as a 4D
  tensor and packed into 256x128 panels, plus a 4D sub-tensor
  (48,64,40,56) of outer sizes (64,80,48,64) with perm (1,3,0,2).
* ``batch_problems`` -- thousands of uneven transposes (N 2..5, element counts
  log-uniform 1Ki..4Mi, FP32/BF16, beta in {0, 0.5}).
* ``serving_requests`` -- a Poisson arrival stream of mixed requests.
* ``complex_cases`` -- the paper's complex types (section 2.1: c, z and the
  mixed cz, zc), N = 2..6, 256 MiB per single-complex input tensor, complex
  alpha, beta in {0, complex}.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np

DTYPE_BYTES = {"f32": 4, "f64": 8, "bf16": 2, "e4m3": 1, "c64": 8, "c128": 16}


@dataclass
class Problem:
    perm: tuple
    sizes: tuple
    dtype_in: str = "f32"
    dtype_out: str = "f32"
    alpha: float | complex = 1.0
    beta: float | complex = 0.0
    outer_a: tuple | None = None
    outer_b: tuple | None = None
    tag: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(np.prod(self.sizes, dtype=np.int64))

    @property
    def sizes_b(self) -> tuple:
        return tuple(self.sizes[p] for p in self.perm)

    @property
    def vol_a(self) -> int:
        return int(np.prod(self.outer_a if self.outer_a else self.sizes, dtype=np.int64))

    @property
    def vol_b(self) -> int:
        return int(np.prod(self.outer_b if self.outer_b else self.sizes_b, dtype=np.int64))

    def algorithmic_bytes(self) -> int:
        """n*(s_A + s_B) for beta == 0, n*(s_A + 2 s_B) otherwise."""
        sa, sb = DTYPE_BYTES[self.dtype_in], DTYPE_BYTES[self.dtype_out]
        return self.n * (sa + (2 * sb if self.beta != 0 else sb))


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def near_equal_sizes(N: int, target: int, g: np.random.Generator, lo=0.85, hi=1.15,
                     tol=0.01, min_size=2) -> tuple:
    """Sizes s_k = round(target^(1/N) * u_k), u_k ~ U[lo, hi], each >= min_size,
    the last one adjusted so that the product is within +-tol of target."""
    base = target ** (1.0 / N)
    for _ in range(1000):
        s = [max(min_size, int(round(base * g.uniform(lo, hi)))) for _ in range(N)]
        rest = int(np.prod(s[:-1], dtype=np.int64))
        s[-1] = max(min_size, int(round(target / rest)))
        n = rest * s[-1]
        if abs(n / target - 1.0) <= tol:
            return tuple(s)
    raise RuntimeError("could not draw sizes")


def random_perm(N: int, g: np.random.Generator, keep0: bool | None = None) -> tuple:
    """A random non-identity permutation; keep0 forces perm[0]==0 (True) or
    perm[0]!=0 (False)."""
    ident = tuple(range(N))
    for _ in range(10000):
        p = tuple(int(x) for x in g.permutation(N))
        if p == ident:
            continue
        if keep0 is True and p[0] != 0:
            continue
        if keep0 is False and p[0] == 0:
            continue
        return p
    raise RuntimeError("no such permutation")


def single_4d() -> Problem:
    return Problem(perm=(2, 0, 3, 1), sizes=(32, 40, 24, 36), tag="single4d")


def sweep_perms(N: int, g: np.random.Generator, count: int = 8) -> list:
    """`count` seeded perms for one N: distinct where enough exist, at least one
    keeping index 0 and one moving it (N >= 3); repeats (with new size draws)
    fill up when fewer than `count` non-identity perms exist."""
    ident = tuple(range(N))
    allp = [p for p in itertools.permutations(range(N)) if p != ident]
    if len(allp) <= count:
        out = list(allp)
        while len(out) < count:
            out.append(allp[int(g.integers(len(allp)))])
        return out
    out = [random_perm(N, g, keep0=True), random_perm(N, g, keep0=False)]
    while len(out) < count:
        p = random_perm(N, g)
        if p not in out:
            out.append(p)
    return out


def sweep_cases(seed: int = 1, target: int = 1 << 26, Ns=(2, 3, 4, 5, 6), perms_per_n=8,
                dtypes=("f32", "f64"), betas=(0.0, 0.4), alpha=1.7) -> list:
    g = rng(seed)
    cases = []
    for N in Ns:
        for pi, perm in enumerate(sweep_perms(N, g, perms_per_n)):
            sizes = near_equal_sizes(N, target, g)
            for dt in dtypes:
                for beta in betas:
                    cases.append(Problem(perm=perm, sizes=sizes, dtype_in=dt, dtype_out=dt,
                                         alpha=alpha, beta=beta, tag=f"N{N}p{pi}"))
    return cases


def pow2_cases(seed: int = 2, log2n: int = 26, Ns=(2, 3, 4, 5, 6), perms_per_n=2, dtypes=("f32", "f64"),
               alpha=1.7) -> list:
    """The sweep's shapes with power-of-two sizes: 2^log2n elements, the
    exponent split as evenly as possible over the N indices (larger ones
    first); perms_per_n seeded perms per N (one keeping index 0 when N >= 3),
    beta = 0."""
    g = rng(seed)
    cases = []
    for N in Ns:
        e = [log2n // N + (1 if k < log2n % N else 0) for k in range(N)]
        sizes = tuple(1 << x for x in e)
        for pi, perm in enumerate(dict.fromkeys(sweep_perms(N, g, perms_per_n))):
            for dt in dtypes:
                cases.append(Problem(perm=perm, sizes=sizes, dtype_in=dt, dtype_out=dt, alpha=alpha, beta=0.0,
                                     tag=f"P{N}p{pi}"))
    return cases


def packing_cases(out_dtypes=("bf16", "e4m3")) -> list:
    """GEMM packing (section 2.1, Fig. 3: a matrix reinterpreted as a 3D/4D
    tensor whose permutation lays out contiguous panels; Fig. 2: a sub-tensor
    of a larger tensor, described by its outer sizes)."""
    cases = []
    for dt in out_dtypes:
        # 4096x2048 sub-block of an 8192x8192 column-major matrix: m = m1 + 256 m2,
        # k = k1 + 128 k2; B(m1,k1,m2,k2) = contiguous 256x128 panels.
        cases.append(Problem(perm=(0, 2, 1, 3), sizes=(256, 16, 128, 16), dtype_in="f32",
                             dtype_out=dt, outer_a=(256, 32, 128, 64), tag="panel",
                             extra={"matrix": (8192, 8192), "offset": (0, 0)}))
        cases.append(Problem(perm=(0, 2, 1, 3), sizes=(256, 16, 128, 16), dtype_in="f32",
                             dtype_out=dt, outer_a=(256, 32, 128, 64), tag="panel_off",
                             extra={"matrix": (8192, 8192), "offset": (64, 128)}))
        cases.append(Problem(perm=(1, 3, 0, 2), sizes=(48, 64, 40, 56), dtype_in="f32",
                             dtype_out=dt, outer_a=(64, 80, 48, 64), tag="sub4d"))
        # the other panel order, B(m1,k1,k2,m2): panels of one row block of
        # m adjacent (a variant of the Fig. 3 reading)
        cases.append(Problem(perm=(0, 2, 3, 1), sizes=(256, 16, 128, 16), dtype_in="f32",
                             dtype_out=dt, outer_a=(256, 32, 128, 64), tag="panel_alt",
                             extra={"matrix": (8192, 8192), "offset": (0, 0)}))
    return cases


def complex_cases(seed: int = 5, target: int = 1 << 25, Ns=(2, 3, 4, 5, 6), perms_per_n=2,
                  pairs=(("c64", "c64"), ("c128", "c128"), ("c64", "c128"), ("c128", "c64")),
                  alpha=complex(1.7, -0.6), beta=complex(0.4, 0.25)) -> list:
    """Complex transposes (section 2.1: single- and double-complex, and the
    mixed cz / zc): near-equal random sizes with `target` elements (+-1 %),
    perms_per_n seeded perms per N (one keeping index 0 when N >= 3), every
    dtype pair, beta = 0 and beta = `beta` alternating over the pairs."""
    g = rng(seed)
    cases = []
    for N in Ns:
        for pi, perm in enumerate(sweep_perms(N, g, perms_per_n)):
            sizes = near_equal_sizes(N, target, g)
            for qi, (di, do) in enumerate(pairs):
                b = beta if (qi + pi) % 2 else 0.0
                cases.append(Problem(perm=perm, sizes=sizes, dtype_in=di, dtype_out=do, alpha=alpha, beta=b,
                                     tag=f"C{N}p{pi}"))
    return cases


def contraction_cases() -> list:
    """Tensor contractions of the kind TTGT serves (section 1): each a dict of
    integer labels per tensor and one extent per label.
    * ttgt4d: C[a,b,c,d] = A[a,e,b,f] B[f,c,e,d], all extents 48: both
      operands and the result need a transpose (interleaved free labels);
    * ttgt3d: C[a,b,c] = A[d,a,c] B[d,b]: A is already a (transposed) matrix,
      C's free labels are interleaved;
    * matrix: C[a,b] = A[a,k] B[k,b], 4096^3: a plain GEMM, no transpose."""
    return [
        {"tag": "ttgt4d", "modes_a": (0, 4, 1, 5), "modes_b": (5, 2, 4, 3), "modes_c": (0, 1, 2, 3),
         "extents": {0: 48, 1: 48, 2: 48, 3: 48, 4: 48, 5: 48}},
        {"tag": "ttgt3d", "modes_a": (3, 0, 2), "modes_b": (3, 1), "modes_c": (0, 1, 2),
         "extents": {0: 256, 1: 512, 2: 256, 3: 512}},
        {"tag": "matrix", "modes_a": (0, 2), "modes_b": (2, 1), "modes_c": (0, 1),
         "extents": {0: 4096, 1: 4096, 2: 4096}},
    ]


def packed_gemm_cases() -> list:
    """GEMMs whose left operand is a packed (permuted, sub-tensor, BF16)
    panel of an FP32 tensor (section 2.1, Figs. 2-3):
    * subblock: a 4096 x 2048 block of an 8192 x 8192 matrix, N = 4096;
    * transposed: the same extents with A stored K x M;
    * ttgt4d: A[a,e,b,f], all extents 48, packed as (a b) x (e f), N = 2304."""
    return [
        {"tag": "subblock", "perm": (0, 1), "sizes": (4096, 2048), "outer": (8192, 8192), "rank_m": 1, "n": 4096},
        {"tag": "transposed", "perm": (1, 0), "sizes": (2048, 4096), "outer": None, "rank_m": 1, "n": 4096},
        {"tag": "ttgt4d", "perm": (0, 2, 1, 3), "sizes": (48, 48, 48, 48), "outer": None, "rank_m": 2, "n": 2304},
    ]


def batch_problems(count: int = 4096, seed: int = 3, lo_log2=10, hi_log2=22,
                   Nmin=2, Nmax=5) -> list:
    g = rng(seed)
    probs = []
    for i in range(count):
        N = int(g.integers(Nmin, Nmax + 1))
        n_target = int(round(2.0 ** g.uniform(lo_log2, hi_log2)))
        sizes = near_equal_sizes(N, n_target, g, tol=0.05 if n_target > 4096 else 0.25)
        perm = random_perm(N, g)
        dt = "f32" if g.random() < 0.5 else "bf16"
        beta = 0.0 if g.random() < 0.5 else 0.5
        probs.append(Problem(perm=perm, sizes=sizes, dtype_in=dt, dtype_out=dt, alpha=1.0,
                             beta=beta, tag=f"b{i}"))
    return probs


def serving_requests(count: int = 2000, seed: int = 4, rate_per_s: float = 20000.0,
                     lo_bytes=4096, hi_bytes=512 << 20, pack_frac=0.10) -> list:
    """Poisson arrivals; request size log-uniform in bytes of A; N 2..6; dtype
    FP32/FP64/BF16 at 50/20/30 %; 10 % packing requests (outer sizes ~1.25x per
    index, BF16 output).  Returns (arrival_time_s, Problem) pairs."""
    g = rng(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += g.exponential(1.0 / rate_per_s)
        N = int(g.integers(2, 7))
        u = g.random()
        dt = "f32" if u < 0.5 else ("f64" if u < 0.7 else "bf16")
        packing = g.random() < pack_frac
        if packing:
            dt = "f32"
        nbytes = math.exp(g.uniform(math.log(lo_bytes), math.log(hi_bytes)))
        n_target = max(64, int(nbytes / DTYPE_BYTES[dt]))
        sizes = near_equal_sizes(N, n_target, g, tol=0.25 if n_target < 1 << 16 else 0.05)
        perm = random_perm(N, g)
        if packing:
            outer = tuple(int(math.ceil(s * g.uniform(1.2, 1.3))) for s in sizes)
            p = Problem(perm=perm, sizes=sizes, dtype_in="f32", dtype_out="bf16",
                        outer_a=outer, tag=f"r{i}pack")
        else:
            p = Problem(perm=perm, sizes=sizes, dtype_in=dt, dtype_out=dt, tag=f"r{i}")
        out.append((t, p))
    return out


# ---------------------------------------------------------------- data ----

def uniform(n: int, seed: int, dtype=np.float32, lo=-1.0, hi=1.0) -> np.ndarray:
    return rng(seed).uniform(lo, hi, size=n).astype(dtype)


def normal(n: int, seed: int, dtype=np.float32) -> np.ndarray:
    return rng(seed).standard_normal(size=n).astype(dtype)


def bf16_bits_from_f32_trunc(x: np.ndarray) -> np.ndarray:
    """Input generator for BF16 tensors: the upper half of float32 values
    (truncation), which is a valid set of random bf16 inputs."""
    return (np.ascontiguousarray(x, np.float32).view(np.uint32) >> 16).astype(np.uint16)


def tensor_for(dtype: str, n: int, seed: int, dist="uniform") -> np.ndarray:
    """Random buffer of n elements in the storage type of `dtype`
    (float32 / float64 / uint16 for bf16 / uint8 for e4m3)."""
    if dtype == "f64":
        return (uniform(n, seed, np.float64) if dist == "uniform" else normal(n, seed, np.float64))
    x = uniform(n, seed, np.float32) if dist == "uniform" else normal(n, seed, np.float32)
    if dtype == "f32":
        return x
    if dtype == "bf16":
        return bf16_bits_from_f32_trunc(x)
    if dtype == "e4m3":
        return rng(seed).integers(0, 256, size=n, dtype=np.uint8)
    if dtype in ("c64", "c128"):
        # (real, imaginary) pairs, both parts from the same distribution
        parts = (uniform(2 * n, seed, np.float64) if dist == "uniform" else normal(2 * n, seed, np.float64))
        return parts.astype(np.float32 if dtype == "c64" else np.float64).view(STORAGE[dtype])
    raise ValueError(dtype)


STORAGE = {"f32": np.float32, "f64": np.float64, "bf16": np.uint16, "e4m3": np.uint8, "c64": np.complex64,
           "c128": np.complex128}
