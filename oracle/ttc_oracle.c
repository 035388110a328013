/*
 * ttc_oracle.c -- plain, slow, obviously-correct CPU oracle for the tensor
 * permute-scale-add of TTC (Springer, Sankaran, Bientinesi, arXiv 1607.01249).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or constant with the
 * CUDA path.
 *
 * What it computes (paper section 1, Eq. 1):
 *     B[Pi(i0..iN-1)] <- alpha * A[i0..iN-1] + beta * B[Pi(i0..iN-1)]
 * on column-major tensors (section 1, footnote 2: index 0 is stride-1) whose
 * indices may each live inside a larger "outer" extent (section 2.1, Table 1
 * --lda/--ldb, Fig. 2: sub-tensors of larger tensors).
 *
 * Permutation convention (section 2.1, Fig. 2b/2c and Fig. 3): perm[d] names
 * the A index that becomes B's index d, so perm=2,1,0 on A(i0,i1,i2) gives
 * B(i2,i1,i0) and perm=0,2,1 on A(m1,m2,k) gives B(m1,k,m2).
 *
 * The oracle is the definition written out: an odometer over every
 * multi-index i of A in column-major order, offsets from the outer extents,
 * one element at a time.  It never merges indices, never tiles, never
 * vectorises.
 *
 * Readings of points the paper leaves open (each is also listed in the design
 * notes of the repository):
 *  - outer extents of B are given in B's own index order; NULL means dense.
 *  - beta == 0: B is not read (NaN/Inf in B do not propagate).
 *  - alpha == 1, beta == 0, same type in and out: a bit copy.
 *  - compute type is FP64 when A or B is FP64, else FP32; alpha and beta are
 *    rounded once to the compute type.
 *  - FP32 compute evaluates r = fmaf(beta, b, fl32(alpha * a)) and rounds r
 *    once to the output type (RNE).  FP64 compute evaluates
 *    r = fma(beta, b, fl64(alpha * a)).
 *  - FP8 E4M3 outputs (OCP "E4M3FN": no infinities, max 448) take
 *    q = RNE_satfinite(fl32(fl32(alpha*a) / scale)), with scale either given
 *    or scale = fl32(amax / 448), amax = max over non-NaN |fl32(alpha*a)|,
 *    and scale = 1 when amax is 0 or not finite or amax/448 underflows to 0.
 *  - Complex types (section 2.1: single-complex "c", double-complex "z", and
 *    the mixed cz / zc): an element is a (real, imaginary) pair; alpha and
 *    beta are complex.  Compute type: double-complex when A or B is
 *    double-complex, else single-complex; each part of alpha and beta is
 *    rounded once to it.  With alpha = (ar, ai), beta = (br, bi), a = (x, y),
 *    b = (u, v), the parts are evaluated in this order:
 *        re = fl(ar*x), im = fl(ar*y)
 *        if ai != 0:   re = fma(-ai, y, re), im = fma(ai, x, im)
 *        if beta != 0: re = fma(br, u, re),  im = fma(br, v, im)
 *                      if bi != 0: re = fma(-bi, v, re), im = fma(bi, u, im)
 *    then each part is rounded once to B's part type.  Real scalars thus
 *    update each part exactly as a real tensor of that type is updated.
 *
 * Build: plain C99, -O2 -ffp-contract=off (no fused operations other than the
 * explicit fma/fmaf calls), no fast-math.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* dtype codes of the oracle (its own numbering); C64 / C128 are the
 * single- and double-complex types, stored as (real, imaginary) pairs */
enum { OR_F32 = 0, OR_F64 = 1, OR_BF16 = 2, OR_E4M3 = 3, OR_C64 = 4, OR_C128 = 5 };

#define OR_MAXDIM 32

static int elem_size(int dt) {
    switch (dt) {
    case OR_F32: return 4;
    case OR_F64: return 8;
    case OR_BF16: return 2;
    case OR_E4M3: return 1;
    case OR_C64: return 8;
    case OR_C128: return 16;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Number formats, written from their definitions.                     */
/* ------------------------------------------------------------------ */

static float f32_from_bits(uint32_t u) { float f; memcpy(&f, &u, 4); return f; }
static uint32_t bits_from_f32(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }

/* bfloat16 = the upper 16 bits of an IEEE binary32 (1 sign, 8 exponent,
 * 7 fraction bits).  Widening is exact. */
float oracle_bf16_to_f32(uint16_t h) { return f32_from_bits((uint32_t)h << 16); }

/* Round an IEEE binary32 to bfloat16, round-to-nearest, ties-to-even:
 * keep the upper 16 bits; the dropped 16 bits decide.  Above half -> up;
 * exactly half -> up only if the kept part is odd.  Carry out of the
 * fraction into the exponent is the correct behaviour (it reaches +-Inf at
 * the top of the range).  NaN -> the quiet NaN 0x7FC0 with the sign kept. */
uint16_t oracle_bf16_from_f32(float x) {
    uint32_t u = bits_from_f32(x);
    if (isnan(x)) return (uint16_t)(((u >> 16) & 0x8000u) | 0x7FC0u);
    uint32_t keep = u >> 16;
    uint32_t rem = u & 0xFFFFu;
    if (rem > 0x8000u || (rem == 0x8000u && (keep & 1u))) keep += 1u;
    return (uint16_t)keep;
}

/* OCP 8-bit floating point, E4M3 variant: 1 sign, 4 exponent bits (bias 7),
 * 3 fraction bits; exponent field 15 with fraction 7 is NaN, there is no
 * infinity; largest finite 1.75*2^8 = 448; smallest normal 2^-6; subnormals
 * m * 2^-9, m = 1..7. */
float oracle_e4m3_to_f32(uint8_t c) {
    int s = (c >> 7) & 1, e = (c >> 3) & 15, m = c & 7;
    double v;
    if (e == 15 && m == 7) return s ? -NAN : NAN;
    if (e == 0) v = ldexp((double)m, -9);
    else v = ldexp(1.0 + m / 8.0, e - 7);
    return (float)(s ? -v : v);
}

/* binary32 -> E4M3, round-to-nearest-even, saturating to +-448 ("satfinite":
 * anything beyond the largest finite value, infinities included, becomes the
 * largest finite value of that sign).  NaN -> 0x7F (sign kept). */
uint8_t oracle_e4m3_from_f32(float x) {
    uint8_t s = (uint8_t)(signbit(x) ? 0x80 : 0x00);
    if (isnan(x)) return (uint8_t)(s | 0x7F);
    double ax = fabs((double)x);
    if (isinf(ax)) return (uint8_t)(s | 0x7E);
    if (ax == 0.0) return s;
    int E;
    double quantum;
    if (ax < ldexp(1.0, -6)) {
        E = -6;                     /* subnormal range: quantum 2^-9 */
        quantum = ldexp(1.0, -9);
    } else {
        int e2;
        frexp(ax, &e2);             /* ax = f * 2^e2, f in [0.5, 1) */
        E = e2 - 1;                 /* ax in [2^E, 2^(E+1)) */
        quantum = ldexp(1.0, E - 3);
    }
    double mr = ax / quantum;       /* exact: power-of-two scaling */
    double mi = floor(mr);
    double fr = mr - mi;
    if (fr > 0.5 || (fr == 0.5 && fmod(mi, 2.0) == 1.0)) mi += 1.0;
    /* value = mi * quantum; re-encode */
    double v = mi * quantum;
    if (v > 448.0) return (uint8_t)(s | 0x7E);
    if (v < ldexp(1.0, -6)) {
        int m = (int)(v / ldexp(1.0, -9));
        return (uint8_t)(s | m);
    }
    int e2;
    frexp(v, &e2);
    int Ev = e2 - 1;
    int m = (int)(v / ldexp(1.0, Ev - 3)) - 8;
    return (uint8_t)(s | ((Ev + 7) << 3) | m);
}

/* ------------------------------------------------------------------ */
/* Element access                                                      */
/* ------------------------------------------------------------------ */

static double load_as_f64(const void* base, int dt, int64_t off) {
    switch (dt) {
    case OR_F32: return (double)((const float*)base)[off];
    case OR_F64: return ((const double*)base)[off];
    case OR_BF16: return (double)oracle_bf16_to_f32(((const uint16_t*)base)[off]);
    case OR_E4M3: return (double)oracle_e4m3_to_f32(((const uint8_t*)base)[off]);
    }
    return NAN;
}

static float load_as_f32(const void* base, int dt, int64_t off) {
    switch (dt) {
    case OR_F32: return ((const float*)base)[off];
    case OR_BF16: return oracle_bf16_to_f32(((const uint16_t*)base)[off]);
    case OR_E4M3: return oracle_e4m3_to_f32(((const uint8_t*)base)[off]);
    }
    return NAN;
}

/* ------------------------------------------------------------------ */
/* Index arithmetic: the plain column-major definition                 */
/* ------------------------------------------------------------------ */

/* offset = sum_k idx[k] * prod_{j<k} outer[j]  (column-major, fn. 2) */
static int64_t colmajor_offset(int n, const int64_t* idx, const int64_t* outer) {
    int64_t off = 0, stride = 1;
    for (int k = 0; k < n; ++k) {
        off += idx[k] * stride;
        stride *= outer[k];
    }
    return off;
}

/* Validate the problem; fill the outer extents (dense if NULL) and B's
 * sizes.  Returns 0 if valid. */
static int setup(int n, const int* perm, const int64_t* sizes, const int64_t* outerA,
                 const int64_t* outerB, int64_t* oA, int64_t* oB, int64_t* sizesB) {
    if (n < 1 || n > OR_MAXDIM) return 1;
    int seen[OR_MAXDIM] = {0};
    for (int d = 0; d < n; ++d) {
        if (perm[d] < 0 || perm[d] >= n || seen[perm[d]]) return 2;
        seen[perm[d]] = 1;
    }
    for (int k = 0; k < n; ++k) {
        if (sizes[k] < 0) return 3;
        oA[k] = outerA ? outerA[k] : sizes[k];
        if (oA[k] < sizes[k]) return 4;
    }
    for (int d = 0; d < n; ++d) {
        sizesB[d] = sizes[perm[d]];
        oB[d] = outerB ? outerB[d] : sizesB[d];
        if (oB[d] < sizesB[d]) return 4;
    }
    return 0;
}

/* Advance a column-major odometer; returns 0 when it wraps (done). */
static int odometer_next(int n, int64_t* idx, const int64_t* sizes) {
    for (int k = 0; k < n; ++k) {
        if (++idx[k] < sizes[k]) return 1;
        idx[k] = 0;
    }
    return 0;
}

static int64_t volume(int n, const int64_t* s) {
    int64_t v = 1;
    for (int k = 0; k < n; ++k) v *= s[k];
    return v;
}

/* ------------------------------------------------------------------ */
/* Error-free transformations for the FP64 reference value             */
/* (Ogita, Rump, Oishi 2005, "Accurate sum and dot product":           */
/*  TwoSum of Knuth, TwoProduct through FMA).                           */
/* ------------------------------------------------------------------ */

static void two_sum(double a, double b, double* s, double* t) {
    double x = a + b;
    double z = x - a;
    *t = (a - (x - z)) + (b - z);
    *s = x;
}

static void two_prod(double a, double b, double* p, double* e) {
    *p = a * b;
    *e = fma(a, b, -*p);
}

/* alpha*a + beta*b, as accurately as double-double evaluation allows
 * (the result is faithful and in practice correctly rounded). */
static double accurate_axpby(double alpha, double a, double beta, double b) {
    double p, e, q, f, s, t;
    two_prod(alpha, a, &p, &e);
    two_prod(beta, b, &q, &f);
    if (!isfinite(p) || !isfinite(q) || !isfinite(e) || !isfinite(f)) return p + q;
    two_sum(p, q, &s, &t);
    return s + (t + (e + f));
}

/* Compute type: FP64 when either tensor is FP64 (reading 12), else FP32. */
static int compute_is_f64(int dtA, int dtB) { return dtA == OR_F64 || dtB == OR_F64; }

/* ------------------------------------------------------------------ */
/* FP8 scale                                                            */
/* ------------------------------------------------------------------ */

/* amax = max over the sub-tensor of |fl32(alpha_f * a)|, NaN ignored;
 * scale = fl32(amax / 448); scale = 1 when amax is 0, not finite, or the
 * quotient underflows to 0.  Returns the scale, writes amax. */
float oracle_fp8_scale(int n, const int64_t* sizes, const int64_t* outerA, int dtA,
                       double alpha, const void* A, float* amax_out) {
    int64_t oA[OR_MAXDIM], idx[OR_MAXDIM];
    for (int k = 0; k < n; ++k) oA[k] = outerA ? outerA[k] : sizes[k];
    float af = (float)alpha;
    float amax = 0.0f;
    if (volume(n, sizes) > 0) {
        memset(idx, 0, sizeof(idx));
        do {
            float v = af * load_as_f32(A, dtA, colmajor_offset(n, idx, oA));
            float m = fabsf(v);
            if (!isnan(m) && m > amax) amax = m;
        } while (odometer_next(n, idx, sizes));
    }
    if (amax_out) *amax_out = amax;
    if (amax == 0.0f || !isfinite(amax)) return 1.0f;
    float scale = amax / 448.0f;
    if (scale == 0.0f) return 1.0f;
    return scale;
}

/* ------------------------------------------------------------------ */
/* The two oracle entry points                                          */
/* ------------------------------------------------------------------ */

/*
 * oracle_permute: B[Pi(i)] <- alpha*A[i] + beta*B[Pi(i)], written into B in
 * the output dtype, element by element, following the rounding sequence of
 * the readings above.  Only elements of the sub-tensor are written.
 * fp8_scale is used when dtB is E4M3 (the caller computes it, e.g. with
 * oracle_fp8_scale).  Returns 0, or a positive code for an invalid problem.
 */
int oracle_permute(int n, const int* perm, const int64_t* sizes, const int64_t* outerA,
                   const int64_t* outerB, int dtA, int dtB, double alpha, double beta,
                   const void* A, void* B, float fp8_scale) {
    int64_t oA[OR_MAXDIM], oB[OR_MAXDIM], sB[OR_MAXDIM];
    int64_t i[OR_MAXDIM], j[OR_MAXDIM];
    int rc = setup(n, perm, sizes, outerA, outerB, oA, oB, sB);
    if (rc) return rc;
    if (dtB == OR_E4M3 && (beta != 0.0 || dtA == OR_F64)) return 5;
    if (volume(n, sizes) == 0) return 0;
    const int bitcopy = (alpha == 1.0 && beta == 0.0 && dtA == dtB);
    const int c64 = compute_is_f64(dtA, dtB);
    const float af = (float)alpha, bf = (float)beta;
    const int sa = elem_size(dtA), sb = elem_size(dtB);

    memset(i, 0, sizeof(i));
    do {
        for (int d = 0; d < n; ++d) j[d] = i[perm[d]];      /* B's index d is A's index perm[d] */
        int64_t offA = colmajor_offset(n, i, oA);
        int64_t offB = colmajor_offset(n, j, oB);
        char* pb = (char*)B + offB * sb;
        const char* pa = (const char*)A + offA * sa;
        if (bitcopy) {
            memcpy(pb, pa, (size_t)sa);
        } else if (dtB == OR_E4M3) {
            float v = af * load_as_f32(A, dtA, offA);
            float q = v / fp8_scale;
            *(uint8_t*)pb = oracle_e4m3_from_f32(q);
        } else if (c64) {
            double a = load_as_f64(A, dtA, offA);
            double r = alpha * a;
            if (beta != 0.0) r = fma(beta, load_as_f64(B, dtB, offB), r);
            if (dtB == OR_F64) *(double*)pb = r;
            else *(float*)pb = (float)r;                  /* one RN rounding */
        } else {
            float a = load_as_f32(A, dtA, offA);
            float r = af * a;
            if (beta != 0.0) r = fmaf(bf, load_as_f32(B, dtB, offB), r);
            if (dtB == OR_F32) *(float*)pb = r;
            else *(uint16_t*)pb = oracle_bf16_from_f32(r); /* one RNE rounding */
        }
    } while (odometer_next(n, i, sizes));
    return 0;
}

/*
 * oracle_permute_exact: the mathematically exact value alpha_c*a + beta_c*b
 * (alpha_c, beta_c = alpha, beta rounded to the compute type), rounded once
 * to double (FP32/BF16 data: the products are exact in double, so only the
 * final sum rounds; FP64 data: double-double evaluation).  R receives the
 * value and S the tolerance scale max(|alpha_c*a|, |beta_c*b|, |r|), both in
 * B's layout (arrays of prod(outerB) doubles).  B is read only when
 * beta != 0.  No FP8 here: the FP8 code is checked bit for bit against
 * oracle_permute and its error is measured against R from an F32 run.
 */
int oracle_permute_exact(int n, const int* perm, const int64_t* sizes, const int64_t* outerA,
                         const int64_t* outerB, int dtA, int dtB, double alpha, double beta,
                         const void* A, const void* B, double* R, double* S) {
    int64_t oA[OR_MAXDIM], oB[OR_MAXDIM], sB[OR_MAXDIM];
    int64_t i[OR_MAXDIM], j[OR_MAXDIM];
    int rc = setup(n, perm, sizes, outerA, outerB, oA, oB, sB);
    if (rc) return rc;
    if (volume(n, sizes) == 0) return 0;
    const int c64 = compute_is_f64(dtA, dtB);
    const double ac = c64 ? alpha : (double)(float)alpha;
    const double bc = c64 ? beta : (double)(float)beta;

    memset(i, 0, sizeof(i));
    do {
        for (int d = 0; d < n; ++d) j[d] = i[perm[d]];
        int64_t offA = colmajor_offset(n, i, oA);
        int64_t offB = colmajor_offset(n, j, oB);
        double a = load_as_f64(A, dtA, offA);
        double r, s;
        if (beta == 0.0) {
            r = ac * a;   /* FP32/BF16 data: the product is exact; FP64: one rounding */
            s = fabs(r);
        } else {
            double b = load_as_f64(B, dtB, offB);
            r = accurate_axpby(ac, a, bc, b);
            s = fmax(fmax(fabs(ac * a), fabs(bc * b)), fabs(r));
        }
        R[offB] = r;
        S[offB] = s;
    } while (odometer_next(n, i, sizes));
    return 0;
}

/* ------------------------------------------------------------------ */
/* Complex types                                                        */
/* ------------------------------------------------------------------ */

static int is_complex_pair(int dtA, int dtB) {
    return (dtA == OR_C64 || dtA == OR_C128) && (dtB == OR_C64 || dtB == OR_C128);
}

/* the two parts of a complex element, widened exactly to double */
static void load_complex(const void* base, int dt, int64_t off, double* re, double* im) {
    if (dt == OR_C64) {
        const float* q = (const float*)base + 2 * off;
        *re = (double)q[0];
        *im = (double)q[1];
    } else {
        const double* q = (const double*)base + 2 * off;
        *re = q[0];
        *im = q[1];
    }
}

static void store_complex(void* base, int dt, int64_t off, double re, double im) {
    if (dt == OR_C64) {
        float* q = (float*)base + 2 * off;
        q[0] = (float)re;                 /* one RN rounding per part */
        q[1] = (float)im;
    } else {
        double* q = (double*)base + 2 * off;
        q[0] = re;
        q[1] = im;
    }
}

/*
 * oracle_permute_complex: B[Pi(i)] <- alpha*A[i] + beta*B[Pi(i)] for the
 * complex pairs (c->c, z->z, c->z, z->c), alpha = ar + i ai and
 * beta = br + i bi, following the rounding sequence of the reading in the
 * header.  Returns 0, or a positive code for an invalid problem.
 */
int oracle_permute_complex(int n, const int* perm, const int64_t* sizes, const int64_t* outerA,
                           const int64_t* outerB, int dtA, int dtB, double ar, double ai, double br,
                           double bi, const void* A, void* B) {
    int64_t oA[OR_MAXDIM], oB[OR_MAXDIM], sB[OR_MAXDIM];
    int64_t i[OR_MAXDIM], j[OR_MAXDIM];
    int rc = setup(n, perm, sizes, outerA, outerB, oA, oB, sB);
    if (rc) return rc;
    if (!is_complex_pair(dtA, dtB)) return 5;
    if (volume(n, sizes) == 0) return 0;
    const int bitcopy = (ar == 1.0 && ai == 0.0 && br == 0.0 && bi == 0.0 && dtA == dtB);
    const int beta_nz = (br != 0.0 || bi != 0.0);
    const int wide = (dtA == OR_C128 || dtB == OR_C128);
    const float arf = (float)ar, aif = (float)ai, brf = (float)br, bif = (float)bi;
    const int sa = elem_size(dtA);

    memset(i, 0, sizeof(i));
    do {
        for (int d = 0; d < n; ++d) j[d] = i[perm[d]];
        int64_t offA = colmajor_offset(n, i, oA);
        int64_t offB = colmajor_offset(n, j, oB);
        if (bitcopy) {
            memcpy((char*)B + offB * sa, (const char*)A + offA * sa, (size_t)sa);
            continue;
        }
        double x, y, u = 0.0, v = 0.0;
        load_complex(A, dtA, offA, &x, &y);
        if (beta_nz) load_complex(B, dtB, offB, &u, &v);
        if (wide) {
            double re = ar * x, im = ar * y;
            if (ai != 0.0) {
                re = fma(-ai, y, re);
                im = fma(ai, x, im);
            }
            if (beta_nz) {
                re = fma(br, u, re);
                im = fma(br, v, im);
                if (bi != 0.0) {
                    re = fma(-bi, v, re);
                    im = fma(bi, u, im);
                }
            }
            store_complex(B, dtB, offB, re, im);
        } else {
            /* single-complex data: x, y, u, v hold floats exactly */
            const float xf = (float)x, yf = (float)y, uf = (float)u, vf = (float)v;
            float re = arf * xf, im = arf * yf;
            if (aif != 0.0f) {
                re = fmaf(-aif, yf, re);
                im = fmaf(aif, xf, im);
            }
            if (beta_nz) {
                re = fmaf(brf, uf, re);
                im = fmaf(brf, vf, im);
                if (bif != 0.0f) {
                    re = fmaf(-bif, vf, re);
                    im = fmaf(bif, uf, im);
                }
            }
            store_complex(B, dtB, offB, (double)re, (double)im);
        }
    } while (odometer_next(n, i, sizes));
    return 0;
}

/* sum of k products x[t]*y[t], evaluated as if in twice double precision
 * (Ogita, Rump, Oishi 2005, Algorithm Dot2: TwoProduct of every term, the
 * running sum by TwoSum, the error terms added at the end). */
static double dot2(int k, const double* x, const double* y) {
    double p, s, h, r, q;
    two_prod(x[0], y[0], &p, &s);
    for (int t = 1; t < k; ++t) {
        two_prod(x[t], y[t], &h, &r);
        two_sum(p, h, &p, &q);
        s += q + r;
    }
    return p + s;
}

/*
 * oracle_permute_complex_exact: the exact value of alpha_c*a + beta_c*b by
 * the definition of the complex product, (ar + i ai)(x + i y) =
 * (ar x - ai y) + i (ar y + ai x), with alpha_c, beta_c the scalars rounded
 * part by part to the compute type; each part evaluated by Dot2 and rounded
 * to double.  R receives (re, im) and S the tolerance scale of each part (the
 * sum of the absolute values of its products), two doubles per element in
 * B's layout.  B is read only when beta != 0.
 */
int oracle_permute_complex_exact(int n, const int* perm, const int64_t* sizes, const int64_t* outerA,
                                 const int64_t* outerB, int dtA, int dtB, double ar, double ai, double br,
                                 double bi, const void* A, const void* B, double* R, double* S) {
    int64_t oA[OR_MAXDIM], oB[OR_MAXDIM], sB[OR_MAXDIM];
    int64_t i[OR_MAXDIM], j[OR_MAXDIM];
    int rc = setup(n, perm, sizes, outerA, outerB, oA, oB, sB);
    if (rc) return rc;
    if (!is_complex_pair(dtA, dtB)) return 5;
    if (volume(n, sizes) == 0) return 0;
    const int wide = (dtA == OR_C128 || dtB == OR_C128);
    const int beta_nz = (br != 0.0 || bi != 0.0);
    const double arc = wide ? ar : (double)(float)ar, aic = wide ? ai : (double)(float)ai;
    const double brc = wide ? br : (double)(float)br, bic = wide ? bi : (double)(float)bi;

    memset(i, 0, sizeof(i));
    do {
        for (int d = 0; d < n; ++d) j[d] = i[perm[d]];
        int64_t offA = colmajor_offset(n, i, oA);
        int64_t offB = colmajor_offset(n, j, oB);
        double x, y, u = 0.0, v = 0.0;
        load_complex(A, dtA, offA, &x, &y);
        if (beta_nz) load_complex(B, dtB, offB, &u, &v);
        const int k = beta_nz ? 4 : 2;
        const double cre[4] = {arc, -aic, brc, -bic}, vre[4] = {x, y, u, v};
        const double cim[4] = {arc, aic, brc, bic}, vim[4] = {y, x, v, u};
        double sre = 0.0, sim = 0.0;
        for (int t = 0; t < k; ++t) {
            sre += fabs(cre[t] * vre[t]);
            sim += fabs(cim[t] * vim[t]);
        }
        R[2 * offB] = dot2(k, cre, vre);
        R[2 * offB + 1] = dot2(k, cim, vim);
        S[2 * offB] = sre;
        S[2 * offB + 1] = sim;
    } while (odometer_next(n, i, sizes));
    return 0;
}

/* Vector helpers for the tests of the number formats. */
void oracle_bf16_from_f32_n(const float* x, uint16_t* y, int64_t n) {
    for (int64_t k = 0; k < n; ++k) y[k] = oracle_bf16_from_f32(x[k]);
}
void oracle_e4m3_from_f32_n(const float* x, uint8_t* y, int64_t n) {
    for (int64_t k = 0; k < n; ++k) y[k] = oracle_e4m3_from_f32(x[k]);
}
void oracle_e4m3_to_f32_n(const uint8_t* x, float* y, int64_t n) {
    for (int64_t k = 0; k < n; ++k) y[k] = oracle_e4m3_to_f32(x[k]);
}
/* fmaf exposed so that a test can pin it against exact rational arithmetic */
void oracle_fmaf_n(const float* a, const float* b, const float* c, float* y, int64_t n) {
    for (int64_t k = 0; k < n; ++k) y[k] = fmaf(a[k], b[k], c[k]);
}
