/*
 * lcq_oracle.c -- plain, slow, scalar CPU oracle for the guaranteed-error-bound
 * quantizers of Fallin & Burtscher, "Lessons Learned on the Path to Guaranteeing
 * the Error Bound in Lossy Quantizers" (arXiv 2407.15037).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant with the CUDA library; the two are written
 * independently from the same paper and the same numbered readings (R1..R11
 * below), and the tests compare them element by element.
 *
 * Build (done by oracle/build.py):
 *   gcc -std=c11 -O2 -fPIC -shared -ffp-contract=off -mno-fma -fno-fast-math
 *       -frounding-math -fexcess-precision=standard -o liblcq_oracle.so
 *       lcq_oracle.c -lquadmath -lm
 * The no-FMA / no-contraction flags are the paper's Sec. 3.2 fix; every
 * floating-point expression below is one IEEE-754 operation in the data type
 * (float for float32 data, double for float64 data).
 *
 * Readings of points the paper leaves open, numbered R1-R11:
 *  R1  "round to the nearest bin" (Sec. 2.2) = round half to even (rint), and
 *      the range test |q| < maxbin is made on the float q BEFORE converting to
 *      an integer, written so that NaN fails it.  The paper's two-sided integer
 *      test (Sec. 3.3) is kept as well.
 *  R2  ABS bound: the user's bound eb is a double; for float32 data the kernel
 *      compares against eb_T = RD_f32(eb), the largest float <= eb, so a float
 *      comparison can never accept more than the double bound.  Pass iff
 *      |x - recon| <= eb_T (the paper's "> eb => outlier", NaN-safe).
 *  R3  maxbin = 2^30 for ABS/NOA, 2^29 for REL (sign bit folded into the bin).
 *  R4  REL: zero, denormal, Inf, NaN inputs are outliers.  L = log2approx(|x|),
 *      lb = fl(e_T / fl(1 + e_T)), step = 2 lb, inv_l = fl(1/step);
 *      b = rint(fl(L * inv_l)); Lr = fl(b * step); the reconstruction is
 *      valid only if bb = fl(Lr + bias) lies in [1, 2*bias+1) (a normal
 *      exponent field); m = pow2approx(Lr); x' = copysign(m, x).  Accept iff
 *      m/2 <= |x| <= 2m (so d = ||x| - m| is exact by Sterbenz) and
 *      d * sc <= t, t = fl(fl(min(|x|, m) * sc) * chk), chk = fl(e_T (1 - 2^-p)),
 *      t normal, where sc = 2^64 if min(|x|, m) < 2^-62 else 1 (float64:
 *      2^512 below 2^-511); the power-of-two rescale is exact and keeps t out
 *      of the subnormal range.  RN(y chk) <= y e_T for normal results, so this
 *      enforces |x|/(1+eb) <= |x'| <= |x|(1+eb) (Sec. 2.1.2).
 *      Stored bin = 2 b + signbit(x).
 *  R5  float64 REL uses the same construction with 52 mantissa bits, an 11-bit
 *      exponent and bias 1023.
 *  R6  NOA: min and max over FINITE values only; R = RD(max - min) and
 *      eb_abs = RD(eb * R), both in double with rounding toward -inf; then
 *      ABS with eb_abs.  No finite value, or derived constants that are not
 *      finite and normal, make every element an outlier (lossless).  A zero
 *      range is +0 (R is a length; x - x rounded toward -inf would give -0,
 *      and which signed zero is min or max must not matter).
 *  R7  -0 and tiny ABS inputs quantize to bin 0 and decode as +0.
 *  R8  Outlier layout: mask bit (i & 31) of word (i >> 5); payload = raw bits
 *      of the outliers in ascending index order; bins of outliers are 0.
 *  R9  No flush-to-zero / denormals-are-zero anywhere (checked at run time).
 *  R10 One recipe, one answer: the bound admits many bins; parity is defined
 *      against this recipe only.
 *  R11 16-bit inputs (IEEE binary16 "f16", bfloat16 "bf16"; the paper covers
 *      float and double only): every value widens exactly to a float and
 *      takes the float recipe with the float constants of R2/R4/R6, except
 *      that the reconstruction the check of Sec. 3.1 tests is the one the
 *      decoder outputs, the float reconstruction rounded to nearest-even in
 *      the 16-bit format.  REL specials are those of the widened float (an
 *      f16 subnormal is a normal float and is quantized).  Outlier payloads
 *      are the raw 16-bit patterns.
 */
#include <float.h>
#include <fenv.h>
#include <math.h>
#include <stdint.h>
#include <string.h>
#include <quadmath.h>
#include <xmmintrin.h>

#pragma STDC FENV_ACCESS ON

#define LCQO_F32 0
#define LCQO_F64 1
#define LCQO_F16 2  /* IEEE binary16, reading R11 */
#define LCQO_BF16 3 /* bfloat16, reading R11 */
#define LCQO_ABS 0
#define LCQO_REL 1
#define LCQO_NOA 2

#define LCQO_OK 0
#define LCQO_BAD_ARG 1
#define LCQO_BAD_BOUND 2

#define MAXBIN_ABS 1073741824 /* 2^30, reading R3 */
#define MAXBIN_REL 536870912  /* 2^29, reading R3 */

/* Derived constants of one quantization.  Float32 values are held exactly in
 * the double fields. */
typedef struct {
    int32_t dtype;        /* LCQO_F32 / LCQO_F64 / LCQO_F16 / LCQO_BF16 */
    int32_t bound;        /* LCQO_ABS / LCQO_REL / LCQO_NOA */
    int32_t all_outliers; /* NOA without a usable range: store everything */
    int32_t pad;
    double eb;            /* the user's bound */
    double R;             /* NOA: RD(max - min) over finite values */
    double eb_abs;        /* ABS: eb; NOA: RD(eb * R); REL: unused */
    double ebT;           /* ABS/NOA: RD_T(eb_abs); REL: RD_T(eb) */
    double eb2;           /* ABS/NOA: 2 ebT */
    double inv;           /* ABS/NOA: fl_T(1 / eb2) */
    double lb;            /* REL: log-domain half step */
    double step;          /* REL: log-domain step 2 lb */
    double inv_l;         /* REL: fl_T(1 / step) */
    double chk;           /* REL: acceptance factor fl_T(ebT (1 - 2^-p)) */
} lcqo_consts;

/* ------------------------------------------------------------------------ */
/* Floating-point environment                                                */
/* ------------------------------------------------------------------------ */

/* Reading R9: returns 1 iff MXCSR has neither FTZ (bit 15) nor DAZ (bit 6)
 * set and the rounding mode is round-to-nearest. */
int lcqo_fp_env_ok(void) {
    unsigned csr = _mm_getcsr();
    if (csr & 0x8040u) return 0;
    return fegetround() == FE_TONEAREST;
}

/* Directed rounding used for the NOA range (reading R6): each helper is one
 * IEEE operation executed with the rounding mode set toward -infinity. */
static double rd_sub_f64(double a, double b) {
    fesetround(FE_DOWNWARD);
    volatile double va = a, vb = b;
    volatile double r = va - vb;
    fesetround(FE_TONEAREST);
    return r;
}

static double rd_mul_f64(double a, double b) {
    fesetround(FE_DOWNWARD);
    volatile double va = a, vb = b;
    volatile double r = va * vb;
    fesetround(FE_TONEAREST);
    return r;
}

/* RD_f32(d): the largest float <= d (reading R2). */
static float rd_f32(double d) {
    fesetround(FE_DOWNWARD);
    volatile double vd = d;
    volatile float r = (float)vd;
    fesetround(FE_TONEAREST);
    return r;
}

static uint32_t f32_bits(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }
static float f32_from(uint32_t u) { float f; memcpy(&f, &u, 4); return f; }
static uint64_t f64_bits(double f) { uint64_t u; memcpy(&u, &f, 8); return u; }
static double f64_from(uint64_t u) { double f; memcpy(&f, &u, 8); return f; }

static int dtype_ok(int dtype) { return dtype >= LCQO_F32 && dtype <= LCQO_BF16; }
static int is_16bit(int dtype) { return dtype == LCQO_F16 || dtype == LCQO_BF16; }

/* ------------------------------------------------------------------------ */
/* 16-bit binary formats (reading R11): sign bit 15, then an exponent field  */
/* of 15 - fb bits with bias `bias`, then fb fraction bits.  binary16:       */
/* fb = 10, bias 15; bfloat16: fb = 7, bias 127.  Written from the format    */
/* definitions with exact double arithmetic.                                 */
/* ------------------------------------------------------------------------ */
static int fmt_fb(int dtype) { return dtype == LCQO_F16 ? 10 : 7; }
static int fmt_bias(int dtype) { return dtype == LCQO_F16 ? 15 : 127; }

/* The value of a 16-bit pattern as a float (exact: both formats are subsets
 * of binary32).  NaN keeps its sign and fraction bits at the top of the
 * float's fraction. */
static float widen16(uint16_t h, int fb, int bias) {
    const uint32_t eall = (1u << (15 - fb)) - 1u;
    const uint32_t s = (uint32_t)h >> 15, E = ((uint32_t)h >> fb) & eall, f = (uint32_t)h & ((1u << fb) - 1u);
    if (E == eall) return f32_from((s << 31) | 0x7F800000u | (f << (23 - fb)));
    double v = (E == 0u) ? ldexp((double)f, 1 - bias - fb) : ldexp((double)(f + (1u << fb)), (int)E - bias - fb);
    return (float)(s ? -v : v);
}

/* x (not NaN) rounded to nearest, ties to even, in the 16-bit format; raw
 * bits.  Magnitudes whose rounding reaches 2^(emax+1) become infinity. */
static uint16_t round16(float x, int fb, int bias) {
    const uint32_t eall = (1u << (15 - fb)) - 1u;
    const uint16_t sgn = signbit(x) ? 0x8000u : 0u;
    const uint16_t inf = (uint16_t)(sgn | (eall << fb));
    const double a = fabs((double)x);
    if (isinf(a)) return inf;
    if (a == 0.0) return sgn;
    const int emin = 1 - bias, emax = (int)eall - 1 - bias;
    int e;
    frexp(a, &e);
    e -= 1; /* a in [2^e, 2^(e+1)) */
    if (e < emin) e = emin;
    const double ulp = ldexp(1.0, e - fb);
    const double r = rint(a / ulp) * ulp; /* a / ulp exact; rint rounds half to even */
    if (r >= ldexp(1.0, emax + 1)) return inf;
    if (r < ldexp(1.0, emin)) return (uint16_t)(sgn | (uint16_t)(r / ldexp(1.0, emin - fb)));
    frexp(r, &e);
    e -= 1;
    const uint32_t f = (uint32_t)(r / ldexp(1.0, e - fb)) - (1u << fb);
    return (uint16_t)(sgn | (uint16_t)(((uint32_t)(e + bias) << fb) | f));
}

/* The decoder's 16-bit output for a float reconstruction, as a float. */
static float through16(float r, int dtype) {
    return widen16(round16(r, fmt_fb(dtype), fmt_bias(dtype)), fmt_fb(dtype), fmt_bias(dtype));
}

void lcqo_widen16_array(int dtype, const uint16_t* h, float* out, uint64_t n) {
    for (uint64_t i = 0; i < n; i++) out[i] = widen16(h[i], fmt_fb(dtype), fmt_bias(dtype));
}

void lcqo_round16_array(int dtype, const float* x, uint16_t* out, uint64_t n) {
    for (uint64_t i = 0; i < n; i++) out[i] = round16(x[i], fmt_fb(dtype), fmt_bias(dtype));
}

/* ------------------------------------------------------------------------ */
/* log2 / pow2 approximations (Sec. 3.2)                                     */
/* ------------------------------------------------------------------------ */

/* For a positive normal float a = 2^(E-127) (1 + M 2^-23) the approximation
 * is log2approx(a) = E - 127 + M 2^-23, evaluated as ONE float addition of the
 * float 1 + M 2^-23 (exponent field of 1.0, a's mantissa field) and the
 * integer E - 128. */
float lcqo_log2approx_f32(float a) {
    uint32_t u = f32_bits(a);
    int32_t E = (int32_t)((u >> 23) & 0xFFu);
    float one_plus_frac = f32_from(0x3F800000u | (u & 0x007FFFFFu));
    float unbiased = (float)(E - 128);
    return one_plus_frac + unbiased;
}

/* Inverse of the above: with bb = fl(L + 127) in [1, 255) and k = floor(bb),
 * pow2approx(L) = 2^(k-127) (1 + (bb - k)).  The fraction bb - k is read off
 * the mantissa field of the float fl(bb - (k - 1)), which lies in [1, 2) and
 * is exact.  Callers guarantee bb in [1, 255). */
float lcqo_pow2approx_f32(float L) {
    float bb = L + 127.0f;
    int32_t k = (int32_t)bb; /* C truncation; bb >= 1 so this is floor */
    float fr = bb - (float)(k - 1);
    uint32_t out = ((uint32_t)k << 23) | (f32_bits(fr) & 0x007FFFFFu);
    return f32_from(out);
}

/* Reading R5: the float64 analogues (11-bit exponent, bias 1023). */
double lcqo_log2approx_f64(double a) {
    uint64_t u = f64_bits(a);
    int64_t E = (int64_t)((u >> 52) & 0x7FFu);
    double one_plus_frac = f64_from(0x3FF0000000000000ull | (u & 0x000FFFFFFFFFFFFFull));
    double unbiased = (double)(E - 1024);
    return one_plus_frac + unbiased;
}

double lcqo_pow2approx_f64(double L) {
    double bb = L + 1023.0;
    int64_t k = (int64_t)bb;
    double fr = bb - (double)(k - 1);
    uint64_t out = ((uint64_t)k << 52) | (f64_bits(fr) & 0x000FFFFFFFFFFFFFull);
    return f64_from(out);
}

/* ------------------------------------------------------------------------ */
/* Constant derivation                                                       */
/* ------------------------------------------------------------------------ */

static int user_bound_ok(double eb) { return eb > 0.0 && isfinite(eb); }

/* ABS constants for bound eb_abs (Sec. 2.2: multiply by the inverse of twice
 * the bound).  Returns 1 iff every derived constant is finite and normal. */
static int derive_abs(int dtype, double eb_abs, lcqo_consts* c) {
    c->eb_abs = eb_abs;
    if (dtype != LCQO_F64) { /* float32 and the 16-bit formats (R11): float constants */
        float ebT = rd_f32(eb_abs);
        if (fpclassify(ebT) != FP_NORMAL) return 0;
        float eb2 = 2.0f * ebT;
        if (!isfinite(eb2)) return 0;
        float inv = 1.0f / eb2;
        if (fpclassify(inv) != FP_NORMAL) return 0;
        c->ebT = ebT; c->eb2 = eb2; c->inv = inv;
    } else {
        double ebT = eb_abs;
        if (fpclassify(ebT) != FP_NORMAL) return 0;
        double eb2 = 2.0 * ebT;
        if (!isfinite(eb2)) return 0;
        double inv = 1.0 / eb2;
        if (fpclassify(inv) != FP_NORMAL) return 0;
        c->ebT = ebT; c->eb2 = eb2; c->inv = inv;
    }
    return 1;
}

int lcqo_consts_abs(int dtype, double eb, lcqo_consts* c) {
    memset(c, 0, sizeof(*c));
    if (!dtype_ok(dtype)) return LCQO_BAD_ARG;
    c->dtype = dtype; c->bound = LCQO_ABS; c->eb = eb;
    if (!user_bound_ok(eb)) return LCQO_BAD_BOUND;
    return derive_abs(dtype, eb, c) ? LCQO_OK : LCQO_BAD_BOUND;
}

/* Reading R4 (REL constants). */
int lcqo_consts_rel(int dtype, double eb, lcqo_consts* c) {
    memset(c, 0, sizeof(*c));
    if (!dtype_ok(dtype)) return LCQO_BAD_ARG;
    c->dtype = dtype; c->bound = LCQO_REL; c->eb = eb;
    if (!user_bound_ok(eb)) return LCQO_BAD_BOUND;
    if (dtype != LCQO_F64) { /* float32 and the 16-bit formats (R11) */
        float e = rd_f32(eb);
        if (fpclassify(e) != FP_NORMAL) return LCQO_BAD_BOUND;
        float onep = 1.0f + e;
        float lb = e / onep;
        float step = 2.0f * lb;
        float inv_l = 1.0f / step;
        float chk = e * 0.99999988079071044921875f; /* 1 - 2^-23 */
        if (fpclassify(lb) != FP_NORMAL || fpclassify(step) != FP_NORMAL ||
            fpclassify(inv_l) != FP_NORMAL || fpclassify(chk) != FP_NORMAL)
            return LCQO_BAD_BOUND;
        c->ebT = e; c->lb = lb; c->step = step; c->inv_l = inv_l; c->chk = chk;
    } else {
        double e = eb;
        if (fpclassify(e) != FP_NORMAL) return LCQO_BAD_BOUND;
        double onep = 1.0 + e;
        double lb = e / onep;
        double step = 2.0 * lb;
        double inv_l = 1.0 / step;
        double chk = e * 0.99999999999999977795539507496869191527366638183594; /* 1 - 2^-52 */
        if (fpclassify(lb) != FP_NORMAL || fpclassify(step) != FP_NORMAL ||
            fpclassify(inv_l) != FP_NORMAL || fpclassify(chk) != FP_NORMAL)
            return LCQO_BAD_BOUND;
        c->ebT = e; c->lb = lb; c->step = step; c->inv_l = inv_l; c->chk = chk;
    }
    return LCQO_OK;
}

/* Reading R6: the largest and smallest FINITE value of the input (Sec. 2.1.3
 * defines R = x_max - x_min over the input). */
void lcqo_range(int dtype, const void* x, uint64_t n, int32_t* any_finite, double* mn, double* mx) {
    int found = 0;
    double lo = 0.0, hi = 0.0;
    for (uint64_t i = 0; i < n; i++) {
        double v;
        if (dtype == LCQO_F32) v = (double)((const float*)x)[i];
        else if (dtype == LCQO_F64) v = ((const double*)x)[i];
        else v = (double)widen16(((const uint16_t*)x)[i], fmt_fb(dtype), fmt_bias(dtype));
        if (!isfinite(v)) continue;
        if (!found) { lo = v; hi = v; found = 1; continue; }
        if (v < lo) lo = v;
        if (v > hi) hi = v;
    }
    *any_finite = found;
    *mn = lo;
    *mx = hi;
}

int lcqo_consts_noa_from_range(int dtype, double eb, int32_t any_finite, double mn, double mx,
                               lcqo_consts* c) {
    memset(c, 0, sizeof(*c));
    if (!dtype_ok(dtype)) return LCQO_BAD_ARG;
    c->dtype = dtype; c->bound = LCQO_NOA; c->eb = eb;
    if (!user_bound_ok(eb)) return LCQO_BAD_BOUND;
    if (!any_finite) { c->all_outliers = 1; return LCQO_OK; }
    c->R = rd_sub_f64(mx, mn);
    if (c->R == 0.0) c->R = 0.0; /* R6: a zero range is +0 */
    double eb_abs = rd_mul_f64(eb, c->R);
    if (!derive_abs(dtype, eb_abs, c)) {
        c->all_outliers = 1;
        c->ebT = c->eb2 = c->inv = 0.0;
    }
    c->eb_abs = eb_abs;
    return LCQO_OK;
}

int lcqo_consts_noa(int dtype, double eb, const void* x, uint64_t n, lcqo_consts* c) {
    int32_t any;
    double mn, mx;
    if (!dtype_ok(dtype)) { memset(c, 0, sizeof(*c)); return LCQO_BAD_ARG; }
    lcqo_range(dtype, x, n, &any, &mn, &mx);
    return lcqo_consts_noa_from_range(dtype, eb, any, mn, mx, c);
}

/* ------------------------------------------------------------------------ */
/* Per-element quantization: returns 1 and the bin for a quantizable value,  */
/* 0 for an outlier.                                                         */
/* ------------------------------------------------------------------------ */

/* ABS / NOA (Sec. 2.2 bin, Sec. 3.1 double-check, Sec. 3.3 two-sided test). */
static int abs_elem_f32(float x, const lcqo_consts* c, int32_t* bin_out) {
    const float inv = (float)c->inv, eb2 = (float)c->eb2, ebT = (float)c->ebT;
    float q = x * inv;
    if (!(fabsf(q) < (float)MAXBIN_ABS)) return 0;
    int32_t bin = (int32_t)rintf(q);
    if ((bin >= MAXBIN_ABS) || (bin <= -MAXBIN_ABS)) return 0;
    float recon = (float)bin * eb2;
    if (!(fabsf(x - recon) <= ebT)) return 0;
    *bin_out = bin;
    return 1;
}

static int abs_elem_f64(double x, const lcqo_consts* c, int32_t* bin_out) {
    double q = x * c->inv;
    if (!(fabs(q) < (double)MAXBIN_ABS)) return 0;
    int32_t bin = (int32_t)rint(q);
    if ((bin >= MAXBIN_ABS) || (bin <= -MAXBIN_ABS)) return 0;
    double recon = (double)bin * c->eb2;
    if (!(fabs(x - recon) <= c->ebT)) return 0;
    *bin_out = bin;
    return 1;
}

/* REL (Sec. 2.1.2 bound, Sec. 3.2 approximations, reading R4). */
static int rel_elem_f32(float x, const lcqo_consts* c, int32_t* bin_out) {
    const float inv_l = (float)c->inv_l, step = (float)c->step, chk = (float)c->chk;
    uint32_t u = f32_bits(x);
    uint32_t s = u >> 31;
    uint32_t E = (u >> 23) & 0xFFu;
    if (E == 0u || E == 0xFFu) return 0; /* zero, denormal, Inf, NaN */
    float a = fabsf(x);
    float L = lcqo_log2approx_f32(a);
    float q = L * inv_l;
    if (!(fabsf(q) < (float)MAXBIN_REL)) return 0;
    int32_t b = (int32_t)rintf(q);
    if ((b >= MAXBIN_REL) || (b <= -MAXBIN_REL)) return 0;
    float Lr = (float)b * step;
    float bb = Lr + 127.0f;
    if (!(bb >= 1.0f && bb < 255.0f)) return 0;
    float m = lcqo_pow2approx_f32(Lr);
    if (!(a <= 2.0f * m && m <= 2.0f * a)) return 0;
    float d = fabsf(a - m);
    float lo = (a < m) ? a : m;
    float sc = (lo < 0x1p-62f) ? 0x1p64f : 1.0f; /* exact rescale keeps t normal */
    float t = (lo * sc) * chk;
    if (!(t >= FLT_MIN)) return 0;
    if (!(d * sc <= t)) return 0;
    *bin_out = (int32_t)(((uint32_t)b << 1) | s);
    return 1;
}

static int rel_elem_f64(double x, const lcqo_consts* c, int32_t* bin_out) {
    uint64_t u = f64_bits(x);
    uint32_t s = (uint32_t)(u >> 63);
    uint64_t E = (u >> 52) & 0x7FFull;
    if (E == 0u || E == 0x7FFull) return 0;
    double a = fabs(x);
    double L = lcqo_log2approx_f64(a);
    double q = L * c->inv_l;
    if (!(fabs(q) < (double)MAXBIN_REL)) return 0;
    int32_t b = (int32_t)rint(q);
    if ((b >= MAXBIN_REL) || (b <= -MAXBIN_REL)) return 0;
    double Lr = (double)b * c->step;
    double bb = Lr + 1023.0;
    if (!(bb >= 1.0 && bb < 2047.0)) return 0;
    double m = lcqo_pow2approx_f64(Lr);
    if (!(a <= 2.0 * m && m <= 2.0 * a)) return 0;
    double d = fabs(a - m);
    double lo = (a < m) ? a : m;
    double sc = (lo < 0x1p-511) ? 0x1p512 : 1.0; /* exact rescale keeps t normal */
    double t = (lo * sc) * c->chk;
    if (!(t >= DBL_MIN)) return 0;
    if (!(d * sc <= t)) return 0;
    *bin_out = (int32_t)(((uint32_t)b << 1) | s);
    return 1;
}

/* 16-bit ABS / NOA (reading R11): the float recipe of abs_elem_f32 on the
 * widened value; the check tests the decoder's 16-bit reconstruction. */
static int abs_elem_16(uint16_t h, const lcqo_consts* c, int32_t* bin_out) {
    const float inv = (float)c->inv, eb2 = (float)c->eb2, ebT = (float)c->ebT;
    float x = widen16(h, fmt_fb(c->dtype), fmt_bias(c->dtype));
    float q = x * inv;
    if (!(fabsf(q) < (float)MAXBIN_ABS)) return 0;
    int32_t bin = (int32_t)rintf(q);
    if ((bin >= MAXBIN_ABS) || (bin <= -MAXBIN_ABS)) return 0;
    float recon = (float)bin * eb2;
    float r = through16(recon, c->dtype);
    if (!(fabsf(x - r) <= ebT)) return 0;
    *bin_out = bin;
    return 1;
}

/* 16-bit REL (reading R11): rel_elem_f32 on the widened value, accepting the
 * decoder's 16-bit magnitude RN16(m) in place of m. */
static int rel_elem_16(uint16_t h, const lcqo_consts* c, int32_t* bin_out) {
    const float inv_l = (float)c->inv_l, step = (float)c->step, chk = (float)c->chk;
    float x = widen16(h, fmt_fb(c->dtype), fmt_bias(c->dtype));
    uint32_t u = f32_bits(x);
    uint32_t s = u >> 31;
    uint32_t E = (u >> 23) & 0xFFu;
    if (E == 0u || E == 0xFFu) return 0; /* zero, float denormal, Inf, NaN */
    float a = fabsf(x);
    float L = lcqo_log2approx_f32(a);
    float q = L * inv_l;
    if (!(fabsf(q) < (float)MAXBIN_REL)) return 0;
    int32_t b = (int32_t)rintf(q);
    if ((b >= MAXBIN_REL) || (b <= -MAXBIN_REL)) return 0;
    float Lr = (float)b * step;
    float bb = Lr + 127.0f;
    if (!(bb >= 1.0f && bb < 255.0f)) return 0;
    float m = through16(lcqo_pow2approx_f32(Lr), c->dtype);
    if (!(a <= 2.0f * m && m <= 2.0f * a)) return 0;
    float d = fabsf(a - m);
    float lo = (a < m) ? a : m;
    float sc = (lo < 0x1p-62f) ? 0x1p64f : 1.0f;
    float t = (lo * sc) * chk;
    if (!(t >= FLT_MIN)) return 0;
    if (!(d * sc <= t)) return 0;
    *bin_out = (int32_t)(((uint32_t)b << 1) | s);
    return 1;
}

static int quant_elem(const lcqo_consts* c, const void* x, uint64_t i, int32_t* bin) {
    if (c->all_outliers) return 0;
    if (is_16bit(c->dtype)) {
        uint16_t h = ((const uint16_t*)x)[i];
        return (c->bound == LCQO_REL) ? rel_elem_16(h, c, bin) : abs_elem_16(h, c, bin);
    }
    if (c->dtype == LCQO_F32) {
        float v = ((const float*)x)[i];
        return (c->bound == LCQO_REL) ? rel_elem_f32(v, c, bin) : abs_elem_f32(v, c, bin);
    } else {
        double v = ((const double*)x)[i];
        return (c->bound == LCQO_REL) ? rel_elem_f64(v, c, bin) : abs_elem_f64(v, c, bin);
    }
}

/* Reconstruction as the decompressor computes it (ABS: bin * eb2; REL:
 * pow2approx of bin * step with the stored sign). */
static float recon_f32(const lcqo_consts* c, int32_t bin) {
    if (c->bound == LCQO_REL) {
        int32_t s = bin & 1;
        int32_t b = (bin - s) / 2;
        float m = lcqo_pow2approx_f32((float)b * (float)c->step);
        return s ? -m : m;
    }
    return (float)bin * (float)c->eb2;
}

static double recon_f64(const lcqo_consts* c, int32_t bin) {
    if (c->bound == LCQO_REL) {
        int32_t s = bin & 1;
        int32_t b = (bin - s) / 2;
        double m = lcqo_pow2approx_f64((double)b * c->step);
        return s ? -m : m;
    }
    return (double)bin * c->eb2;
}

/* ------------------------------------------------------------------------ */
/* Whole-array quantize / dequantize with outlier compaction (reading R8)    */
/* ------------------------------------------------------------------------ */

/* Returns the number of outliers.  bins[n], mask[ceil(n/32)], payload[cap]
 * (uint32 bits for float32 data, uint64 bits for float64 data, uint16 bits
 * for the 16-bit formats).  Payload
 * writes stop at cap; the count is always complete. */
uint64_t lcqo_quantize(const lcqo_consts* c, const void* x, uint64_t n, int32_t* bins,
                       uint32_t* mask, void* payload, uint64_t cap) {
    uint64_t words = (n + 31u) / 32u;
    for (uint64_t w = 0; w < words; w++) mask[w] = 0u;
    uint64_t count = 0;
    for (uint64_t i = 0; i < n; i++) {
        int32_t bin = 0;
        if (quant_elem(c, x, i, &bin)) {
            bins[i] = bin;
        } else {
            bins[i] = 0;
            mask[i >> 5] |= 1u << (i & 31u);
            if (count < cap) {
                if (c->dtype == LCQO_F32)
                    ((uint32_t*)payload)[count] = ((const uint32_t*)x)[i];
                else if (c->dtype == LCQO_F64)
                    ((uint64_t*)payload)[count] = ((const uint64_t*)x)[i];
                else
                    ((uint16_t*)payload)[count] = ((const uint16_t*)x)[i];
            }
            count++;
        }
    }
    return count;
}

void lcqo_dequantize(const lcqo_consts* c, const int32_t* bins, const uint32_t* mask,
                     const void* payload, uint64_t n, void* out) {
    uint64_t k = 0;
    for (uint64_t i = 0; i < n; i++) {
        int outlier = (mask[i >> 5] >> (i & 31u)) & 1u;
        if (is_16bit(c->dtype)) { /* R11: the float reconstruction, rounded */
            if (outlier) ((uint16_t*)out)[i] = ((const uint16_t*)payload)[k++];
            else ((uint16_t*)out)[i] = round16(recon_f32(c, bins[i]), fmt_fb(c->dtype), fmt_bias(c->dtype));
        } else if (c->dtype == LCQO_F32) {
            if (outlier) ((uint32_t*)out)[i] = ((const uint32_t*)payload)[k++];
            else ((float*)out)[i] = recon_f32(c, bins[i]);
        } else {
            if (outlier) ((uint64_t*)out)[i] = ((const uint64_t*)payload)[k++];
            else ((double*)out)[i] = recon_f64(c, bins[i]);
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Ablations (not the method; reference outputs for the ablation kernels).   */
/* ------------------------------------------------------------------------ */

/* The unprotected ABS quantizer that Sec. 6 (Tables 7-8) compares against:
 * the bin of Sec. 2.2 with the range tests (R1, Sec. 3.3) but without the
 * reconstruct-and-check of Sec. 3.1.  c must hold ABS constants. */
static int abs_elem_unprotected(const lcqo_consts* c, const void* x, uint64_t i, int32_t* bin_out) {
    int32_t bin;
    if (c->dtype == LCQO_F32) {
        float q = ((const float*)x)[i] * (float)c->inv;
        if (!(fabsf(q) < (float)MAXBIN_ABS)) return 0;
        bin = (int32_t)rintf(q);
    } else {
        double q = ((const double*)x)[i] * c->inv;
        if (!(fabs(q) < (double)MAXBIN_ABS)) return 0;
        bin = (int32_t)rint(q);
    }
    if ((bin >= MAXBIN_ABS) || (bin <= -MAXBIN_ABS)) return 0;
    *bin_out = bin;
    return 1;
}

uint64_t lcqo_quantize_unprotected(const lcqo_consts* c, const void* x, uint64_t n, int32_t* bins,
                                   uint32_t* mask, void* payload, uint64_t cap) {
    if (c->dtype != LCQO_F32 && c->dtype != LCQO_F64) return UINT64_MAX; /* float / double only */
    uint64_t words = (n + 31u) / 32u;
    for (uint64_t w = 0; w < words; w++) mask[w] = 0u;
    uint64_t count = 0;
    for (uint64_t i = 0; i < n; i++) {
        int32_t bin = 0;
        if (abs_elem_unprotected(c, x, i, &bin)) {
            bins[i] = bin;
            continue;
        }
        bins[i] = 0;
        mask[i >> 5] |= 1u << (i & 31u);
        if (count < cap) {
            if (c->dtype == LCQO_F32) ((uint32_t*)payload)[count] = ((const uint32_t*)x)[i];
            else ((uint64_t*)payload)[count] = ((const uint64_t*)x)[i];
        }
        count++;
    }
    return count;
}

/* Decoder of the REL variant that uses the math library's exp2 (Sec. 2.3),
 * with THIS host's C library: m = exp2(b * step) for the stored bin 2b + s,
 * sign s.  Positions whose mask bit is set get 0 (outliers not gathered). */
void lcqo_rel_library_recon(int dtype, double step, const int32_t* bins, const uint32_t* mask, uint64_t n,
                            void* out) {
    for (uint64_t i = 0; i < n; i++) {
        int outlier = (mask[i >> 5] >> (i & 31u)) & 1u;
        int32_t s = bins[i] & 1;
        int32_t b = (bins[i] - s) / 2;
        if (dtype == LCQO_F32) {
            float m = outlier ? 0.0f : exp2f((float)b * (float)step);
            ((float*)out)[i] = (s && !outlier) ? -m : m;
        } else {
            double m = outlier ? 0.0 : exp2((double)b * step);
            ((double*)out)[i] = (s && !outlier) ? -m : m;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Exact verifiers of the bounds (Sec. 2.1) -- independent of the recipe.    */
/* An element passes if its reconstruction is bit-identical to the input,    */
/* or both are finite and the bound holds in exact real arithmetic.          */
/* ------------------------------------------------------------------------ */

/* Exact decision of |x - y| <= e for doubles x, y (finite) and e >= 0.
 * Knuth's TwoSum gives s + err == x - y exactly (round to nearest, no
 * overflow).  Since s = RN(s + err): if |s| < e then |s + err| <= e; if
 * |s| > e then |s + err| > e; if |s| == e the sign of err decides. */
static int abs_diff_le(double x, double y, double e) {
    double a = x, b = -y;
    double s = a + b;
    if (!isfinite(s)) return 0; /* |x - y| exceeds DBL_MAX >= e */
    double bp = s - a;
    double ap = s - bp;
    double db = b - bp;
    double da = a - ap;
    double err = da + db;
    if (s == 0.0) return 1; /* then err == 0 and x == y */
    double sa = fabs(s);
    double ea = (s > 0.0) ? err : -err;
    if (sa < e) return 1;
    if (sa > e) return 0;
    return ea <= 0.0;
}

static int same_bits(int dtype, const void* x, const void* y, uint64_t i) {
    if (dtype == LCQO_F32) return ((const uint32_t*)x)[i] == ((const uint32_t*)y)[i];
    if (dtype == LCQO_F64) return ((const uint64_t*)x)[i] == ((const uint64_t*)y)[i];
    return ((const uint16_t*)x)[i] == ((const uint16_t*)y)[i];
}

static double load_as_f64(int dtype, const void* p, uint64_t i) {
    if (dtype == LCQO_F32) return (double)((const float*)p)[i];
    if (dtype == LCQO_F64) return ((const double*)p)[i];
    return (double)widen16(((const uint16_t*)p)[i], fmt_fb(dtype), fmt_bias(dtype));
}

/* Number of elements violating |x - x'| <= eb (ABS, Sec. 2.1.1; NOA uses
 * eb = eps * R, Sec. 2.1.3). */
uint64_t lcqo_verify_abs(int dtype, const void* x, const void* xr, uint64_t n, double eb) {
    uint64_t bad = 0;
    for (uint64_t i = 0; i < n; i++) {
        if (same_bits(dtype, x, xr, i)) continue;
        double a = load_as_f64(dtype, x, i), b = load_as_f64(dtype, xr, i);
        if (!isfinite(a) || !isfinite(b) || !abs_diff_le(a, b, eb)) bad++;
    }
    return bad;
}

/* Exact decision of |x|/(1+eps) <= |x'| <= |x|(1+eps) with equal signs
 * (Sec. 2.1.2), for 0 < eps < 2^50.  With a = |x| and m = |x'| it is
 * a - m <= m eps and m - a <= a eps.  If max/min >= 2^60 the bound fails
 * outright; otherwise a - m is exact in binary128 (at most 113 bits), and so
 * are the products m eps, a eps (at most 106 bits). */
static int rel_ok(double x, double xr, double eps) {
    if (!isfinite(x) || !isfinite(xr)) return 0;
    if (x == 0.0 || xr == 0.0) return 0; /* a zero must be reproduced exactly */
    if (signbit(x) != signbit(xr)) return 0;
    __float128 a = (__float128)fabs(x), m = (__float128)fabs(xr);
    __float128 two60 = 1152921504606846976.0Q; /* 2^60 */
    if (a >= m * two60 || m >= a * two60) return 0;
    __float128 e = (__float128)eps;
    __float128 D = a - m;
    return (D <= m * e) && (-D <= a * e);
}

uint64_t lcqo_verify_rel(int dtype, const void* x, const void* xr, uint64_t n, double eps) {
    if (!(eps > 0.0 && eps < 1125899906842624.0)) return UINT64_MAX; /* 2^50 */
    uint64_t bad = 0;
    for (uint64_t i = 0; i < n; i++) {
        if (same_bits(dtype, x, xr, i)) continue;
        if (!rel_ok(load_as_f64(dtype, x, i), load_as_f64(dtype, xr, i), eps)) bad++;
    }
    return bad;
}

/* ------------------------------------------------------------------------ */
/* Sweep over float32 bit patterns [start, start + count): quantize each,    */
/* reconstruct it, and check the bound exactly (the exhaustive run of Sec. 6 */
/* at several bounds).  out[0] = outliers, out[1] = violations,              */
/* out[2] = inliers whose reconstruction is not bit-exact (information).     */
/* ------------------------------------------------------------------------ */
void lcqo_sweep_f32(const lcqo_consts* c, uint64_t start, uint64_t count, double eb_verify,
                    uint64_t* out) {
    uint64_t outl = 0, bad = 0, inexact = 0;
    if (c->dtype != LCQO_F32) { out[0] = out[1] = out[2] = UINT64_MAX; return; }
    for (uint64_t i = 0; i < count; i++) {
        uint32_t u = (uint32_t)(start + i);
        float x = f32_from(u);
        int32_t bin = 0;
        float xr;
        if (quant_elem(c, &x, 0, &bin)) {
            xr = recon_f32(c, bin);
        } else {
            xr = x;
            outl++;
        }
        if (f32_bits(xr) == u) continue;
        inexact++;
        int ok;
        if (c->bound == LCQO_REL) ok = rel_ok((double)x, (double)xr, eb_verify);
        else ok = isfinite(x) && isfinite(xr) && abs_diff_le((double)x, (double)xr, eb_verify);
        if (!ok) bad++;
    }
    out[0] = outl;
    out[1] = bad;
    out[2] = inexact;
}

/* Array forms of the Sec. 3.2 approximations, so that the tests can check
 * them against their closed forms over large ranges of inputs. */
void lcqo_log2approx_f32_array(const float* a, float* out, uint64_t n) {
    for (uint64_t i = 0; i < n; i++) out[i] = lcqo_log2approx_f32(a[i]);
}

void lcqo_pow2approx_f32_array(const float* L, float* out, uint64_t n) {
    for (uint64_t i = 0; i < n; i++) out[i] = lcqo_pow2approx_f32(L[i]);
}

void lcqo_log2approx_f64_array(const double* a, double* out, uint64_t n) {
    for (uint64_t i = 0; i < n; i++) out[i] = lcqo_log2approx_f64(a[i]);
}

void lcqo_pow2approx_f64_array(const double* L, double* out, uint64_t n) {
    for (uint64_t i = 0; i < n; i++) out[i] = lcqo_pow2approx_f64(L[i]);
}
