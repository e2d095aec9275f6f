// lcq_device.cuh -- device-side building blocks of liblcq: per-value quantize /
// verify / reconstruct recipes (one IEEE operation per step, explicit
// round-to-nearest intrinsics, so nothing can be contracted into an FMA), the
// workspace head and the end-of-launch bookkeeping.
//
// Method: Fallin & Burtscher, arXiv 2407.15037.  ABS bin (Sec. 2.2), the
// reconstruct-and-check step (Sec. 3.1), IEEE-only arithmetic (Sec. 3.2), the
// log2/pow2 approximations for REL (Sec. 3.2), the two-sided bin-range test
// (Sec. 3.3).  Points the paper leaves open are settled as follows:
//   rounding to a bin is round-half-even; the range test |q| < maxbin runs on
//   the floating-point q before any integer conversion; maxbin = 2^30 for
//   ABS/NOA and 2^29 for REL; for float32 data the ABS threshold is the
//   largest float not above the user's double bound; REL treats zero,
//   denormals, Inf and NaN as outliers and accepts a reconstruction m of
//   a = |x| iff m/2 <= a <= 2m and |a - m| * sc <= RN(RN(min(a, m) * sc) * chk)
//   with that product normal, chk = RN(eb_T (1 - 2^-p)) and sc an exact
//   power-of-two rescale for tiny values; the REL bin stores 2b + signbit.
#pragma once

#include <cfloat>
#include <cstdint>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "../../include/lcq.h"

namespace lcq {

constexpr int32_t kMaxBinAbs = 1 << 30;
constexpr int32_t kMaxBinRel = 1 << 29;

// Kernel modes besides LCQ_ABS (also used for NOA) and LCQ_REL: the two
// ablations of the paper's experiments.  kModeAbsNoCheck is ABS without the
// reconstruct-and-check step (the unprotected quantizer of Sec. 6, Tables 7
// and 8); kModeRelLib is REL with the CUDA math library's log2 / exp2 in
// place of the bit-level approximations (the library variant of Sec. 2.3 and
// Tables 4-6), still double-checked on the device.
constexpr int kModeAbsNoCheck = 3;
constexpr int kModeRelLib = 4;

// ---------------------------------------------------------------------------
// Type traits: every arithmetic step is a single correctly rounded IEEE op.
// ---------------------------------------------------------------------------
template <typename T>
struct Ty;

template <>
struct Ty<float> {
    using U = uint32_t;
    using C = float;  // arithmetic type
    using K = uint32_t;  // order key of the NOA range
    static constexpr uint32_t kDtype = LCQ_F32;
    static constexpr int kP = 23;
    static constexpr int kBias = 127;
    static constexpr U kExpAll = 0xFFu;
    static constexpr U kMant = 0x007FFFFFu;
    static constexpr U kOneBits = 0x3F800000u;
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ int32_t rint_i(float a) { return __float2int_rn(a); }
    static __device__ __forceinline__ int64_t trunc_i(float a) { return __float2int_rz(a); }
    static __device__ __forceinline__ float from_i(int32_t a) { return __int2float_rn(a); }
    static __device__ __forceinline__ float from_i64(int64_t a) { return __int2float_rn((int)a); }
    static __device__ __forceinline__ U bits(float a) { return __float_as_uint(a); }
    static __device__ __forceinline__ float from_bits(U u) { return __uint_as_float(u); }
    static __device__ __forceinline__ float fabs_(float a) { return fabsf(a); }
    static __device__ __forceinline__ float nmin() { return FLT_MIN; }
    static __device__ __forceinline__ float one_minus_ulp() { return 0x1.fffffcp-1f; }  // 1 - 2^-23
    static __device__ __forceinline__ float tiny() { return 0x1p-62f; }
    static __device__ __forceinline__ float rescale() { return 0x1p64f; }
    static __device__ __forceinline__ float top_bb() { return 255.0f; }
    static __device__ __forceinline__ float bias_f() { return 127.0f; }
    static __device__ __forceinline__ double to_f64(float a) { return (double)a; }
};

template <>
struct Ty<double> {
    using U = uint64_t;
    using C = double;
    using K = uint64_t;
    static constexpr uint32_t kDtype = LCQ_F64;
    static constexpr int kP = 52;
    static constexpr int kBias = 1023;
    static constexpr U kExpAll = 0x7FFull;
    static constexpr U kMant = 0x000FFFFFFFFFFFFFull;
    static constexpr U kOneBits = 0x3FF0000000000000ull;
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ int32_t rint_i(double a) { return __double2int_rn(a); }
    static __device__ __forceinline__ int64_t trunc_i(double a) { return __double2ll_rz(a); }
    static __device__ __forceinline__ double from_i(int32_t a) { return __int2double_rn(a); }
    static __device__ __forceinline__ double from_i64(int64_t a) { return __ll2double_rn(a); }
    static __device__ __forceinline__ U bits(double a) { return (U)__double_as_longlong(a); }
    static __device__ __forceinline__ double from_bits(U u) { return __longlong_as_double((long long)u); }
    static __device__ __forceinline__ double fabs_(double a) { return fabs(a); }
    static __device__ __forceinline__ double nmin() { return DBL_MIN; }
    static __device__ __forceinline__ double one_minus_ulp() { return 0x1.ffffffffffffep-1; }  // 1 - 2^-52
    static __device__ __forceinline__ double tiny() { return 0x1p-511; }
    static __device__ __forceinline__ double rescale() { return 0x1p512; }
    static __device__ __forceinline__ double top_bb() { return 2047.0; }
    static __device__ __forceinline__ double bias_f() { return 1023.0; }
    static __device__ __forceinline__ double to_f64(double a) { return a; }
};

// 16-bit storage formats (IEEE binary16 and bfloat16).  The paper works in
// float and double; here a 16-bit value widens exactly to a float, takes the
// float recipe, and the check of Sec. 3.1 tests the decoder's output: the
// float reconstruction rounded to nearest-even in the 16-bit format.  The
// structs hold raw bit patterns; all arithmetic is float32.
struct f16s {
    uint16_t u;
    __host__ __device__ constexpr f16s(int z = 0) : u((uint16_t)z) {}
};
struct bf16s {
    uint16_t u;
    __host__ __device__ constexpr bf16s(int z = 0) : u((uint16_t)z) {}
};

template <typename S, uint32_t DT, int P, uint16_t EALL>
struct Ty16 {
    using U = uint16_t;
    using C = float;
    using K = uint32_t;  // 16-bit order keys, widened for the warp shuffles
    static constexpr uint32_t kDtype = DT;
    static constexpr int kP = P;
    static constexpr U kExpAll = EALL;
    static __device__ __forceinline__ U bits(S a) { return a.u; }
    static __device__ __forceinline__ S from_bits(U u) { return S((int)u); }
};

template <>
struct Ty<f16s> : Ty16<f16s, LCQ_F16, 10, 0x1F> {
    static __device__ __forceinline__ float widen(f16s a) { return __half2float(__ushort_as_half(a.u)); }
    static __device__ __forceinline__ f16s narrow(float x) {
        return f16s((int)__half_as_ushort(__float2half_rn(x)));
    }
    static __device__ __forceinline__ double to_f64(f16s a) { return (double)widen(a); }
    static __device__ __forceinline__ void widen4(const f16s h[4], float v[4]) {
        const float2 a = __half22float2(__halves2half2(__ushort_as_half(h[0].u), __ushort_as_half(h[1].u)));
        const float2 b = __half22float2(__halves2half2(__ushort_as_half(h[2].u), __ushort_as_half(h[3].u)));
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
};

template <>
struct Ty<bf16s> : Ty16<bf16s, LCQ_BF16, 7, 0xFF> {
    static __device__ __forceinline__ float widen(bf16s a) { return __uint_as_float((uint32_t)a.u << 16); }
    static __device__ __forceinline__ bf16s narrow(float x) {
        return bf16s((int)__bfloat16_as_ushort(__float2bfloat16_rn(x)));
    }
    static __device__ __forceinline__ double to_f64(bf16s a) { return (double)widen(a); }
    static __device__ __forceinline__ void widen4(const bf16s h[4], float v[4]) {
        for (int k = 0; k < 4; k++) v[k] = widen(h[k]);
    }
};

// Arithmetic type of a storage type: float for float and the 16-bit formats.
template <typename T>
using CT = typename Ty<T>::C;

template <typename T>
__host__ __device__ constexpr bool is16() { return sizeof(T) == 2; }

// ---------------------------------------------------------------------------
// Exact replacements for conversions (the float<->int conversions run on a
// slow pipe).  Each returns exactly what the conversion it replaces returns:
//   round_small(q): for |q| < 2^22 (float) / 2^51 (double), t = RN(q + 1.5 2^p)
//     lies in one binade with unit spacing, so t - 1.5 2^p = rint(q) (ties to
//     even, as 1.5 2^p is even) exactly, and the bit difference of t and
//     1.5 2^p is that integer;
//   floor_bb(bb): for 0 <= bb < 2^p, RZ(bb + 2^p) = 2^p + floor(bb), exactly;
//   int_to_float_small(i): for |i| < 2^22, the float with bits
//     bits(1.5 2^23) + i is 1.5 2^23 + i, so subtracting 1.5 2^23 gives i.
// ---------------------------------------------------------------------------
struct Rounded {
    int32_t i;  // the integer
    float f32;  // the same integer as a float (float path)
};

__device__ __forceinline__ bool round_small_f32(float q, int32_t& i, float& f) {
    if (!(fabsf(q) < 0x1p22f)) return false;
    const float t = __fadd_rn(q, 0x1.8p23f);
    i = __float_as_int(t) - 0x4B400000;
    f = __fsub_rn(t, 0x1.8p23f);
    return true;
}

__device__ __forceinline__ void round_any_f32(float q, int32_t& i, float& f) {
    if (!round_small_f32(q, i, f)) {
        i = __float2int_rn(q);
        f = __int2float_rn(i);
    }
}

__device__ __forceinline__ void round_any_f64(double q, int32_t& i, double& f) {
    // |q| < 2^30 < 2^51 always holds here
    const double t = __dadd_rn(q, 0x1.8p52);
    i = (int32_t)(__double_as_longlong(t) - 0x4338000000000000ll);
    f = __dsub_rn(t, 0x1.8p52);
}

__device__ __forceinline__ float int_to_float_f32(int32_t i) {
    if (i > -(1 << 22) && i < (1 << 22)) return __fsub_rn(__int_as_float(0x4B400000 + i), 0x1.8p23f);
    return __int2float_rn(i);
}

__device__ __forceinline__ double int_to_float_f64(int32_t i) {
    return __dsub_rn(__longlong_as_double(0x4338000000000000ll + i), 0x1.8p52);
}

// Constants of one quantization, in the data type.
template <typename T>
struct Consts {
    T ebT;     // ABS/NOA: threshold eb_T; REL: eb_T
    T scale;   // ABS/NOA: eb2; REL: step
    T inv;     // ABS/NOA: 1/eb2; REL: 1/step
    T chk;     // REL acceptance factor
    uint32_t all_outliers;
    // float64 REL: the acceptance test is certain to pass for a normal |x|
    // with biased exponent >= cert_emin whose mantissa field M satisfies
    // cert_w <= M < 2^52 - cert_w (see rel_quant_f64); cert_w = 0: never.
    uint32_t cert_emin;
    uint64_t cert_w;
};

template <typename T>
__device__ __forceinline__ Consts<T> consts_from_header(const lcq_header* h) {
    using U = typename Ty<T>::U;
    Consts<T> c;
    c.ebT = Ty<T>::from_bits((U)h->ebT_bits);
    c.scale = Ty<T>::from_bits((U)h->scale_bits);
    c.inv = Ty<T>::from_bits((U)h->inv_bits);
    c.chk = Ty<T>::from_bits((U)h->chk_bits);
    c.all_outliers = h->mode;
    c.cert_emin = 0;
    c.cert_w = 0;
    return c;
}

// ---------------------------------------------------------------------------
// Per-value recipes
// ---------------------------------------------------------------------------

// Per-type rounding / conversion helpers used by the recipes below.
template <typename T>
struct Cv;
template <>
struct Cv<float> {
    static __device__ __forceinline__ void round(float q, int32_t& i, float& f) { round_any_f32(q, i, f); }
    static __device__ __forceinline__ float from_int(int32_t i) { return int_to_float_f32(i); }
    // floor(bb) for 1 <= bb < 255, as integer and as float: RZ(bb + 2^23)
    static __device__ __forceinline__ void floor_bb(float bb, int32_t& k, float& kf) {
        const float t = __fadd_rz(bb, 0x1p23f);
        k = __float_as_int(t) - 0x4B000000;
        kf = __fsub_rn(t, 0x1p23f);
    }
    // (float)(E - 128) for a biased exponent 1 <= E <= 254
    static __device__ __forceinline__ float unbias(uint32_t E) {
        return __fsub_rn(__uint_as_float(0x4B000000u | E), 0x1.00010p23f);  // 2^23 + 128
    }
};
template <>
struct Cv<double> {
    static __device__ __forceinline__ void round(double q, int32_t& i, double& f) { round_any_f64(q, i, f); }
    static __device__ __forceinline__ double from_int(int32_t i) { return int_to_float_f64(i); }
    static __device__ __forceinline__ void floor_bb(double bb, int32_t& k, double& kf) {
        const double t = __dadd_rz(bb, 0x1p52);
        k = (int32_t)(__double_as_longlong(t) - 0x4330000000000000ll);
        kf = __dsub_rn(t, 0x1p52);
    }
    // (double)(E - 1024) for a biased exponent 1 <= E <= 2046
    static __device__ __forceinline__ double unbias(uint64_t E) {
        return __dsub_rn(__longlong_as_double((long long)(0x4330000000000000ull | E)), 0x1.0000000000400p52);
    }
};

// ABS / NOA: bin = rint(x * inv) (Sec. 2.2); reconstruct and check (Sec. 3.1);
// two-sided range test (Sec. 3.3).  Returns false for an outlier.
// CHECK = false drops the reconstruct-and-check step (the unprotected ablation).
template <typename T, bool CHECK = true>
__device__ __forceinline__ bool abs_quant(T x, const Consts<T>& c, int32_t& bin) {
    using F = Ty<T>;
    const T q = F::mul(x, c.inv);
    if (!(F::fabs_(q) < T(kMaxBinAbs))) return false;
    int32_t b;
    T bf;
    Cv<T>::round(q, b, bf);  // b = rint(q), bf = (T)b
    // Sec. 3.3: (b >= maxbin) || (b <= -maxbin), as one unsigned comparison
    if ((uint32_t)(b + (kMaxBinAbs - 1)) > (uint32_t)(2 * (kMaxBinAbs - 1))) return false;
    if constexpr (CHECK) {
        const T recon = F::mul(bf, c.scale);
        if (!(F::fabs_(F::sub(x, recon)) <= c.ebT)) return false;
    }
    bin = b;
    return true;
}

template <typename T>
__device__ __forceinline__ T abs_recon(int32_t bin, const Consts<T>& c) {
    return Ty<T>::mul(Cv<T>::from_int(bin), c.scale);
}

// log2approx (Sec. 3.2): one addition of the float 1.mantissa and E - (bias+1).
template <typename T>
__device__ __forceinline__ T log2approx(typename Ty<T>::U u) {
    using F = Ty<T>;
    const typename F::U E = (u >> F::kP) & F::kExpAll;
    const T one_frac = F::from_bits(F::kOneBits | (u & F::kMant));
    return F::add(one_frac, Cv<T>::unbias(E));
}

// pow2approx (Sec. 3.2) of bb = RN(Lr + bias), bb in [1, 2 bias + 1):
// 2^(k - bias) (1 + bb - k), k = floor(bb); the fraction is the mantissa of
// the float bb - (k - 1), which lies in [1, 2) and is exact.
template <typename T>
__device__ __forceinline__ typename Ty<T>::U pow2approx_bits(T bb) {
    using F = Ty<T>;
    using U = typename F::U;
    int32_t k;
    T kf;
    Cv<T>::floor_bb(bb, k, kf);
    const T fr = F::sub(bb, F::sub(kf, T(1)));
    return ((U)k << F::kP) | (F::bits(fr) & F::kMant);
}

// REL acceptance of a reconstruction m (normal, positive) of a = |x|:
// m/2 <= a <= 2m, then |a - m| (exact by Sterbenz) <= RN(min(a, m) * chk),
// that product normal; tiny values are rescaled by an exact power of two.
template <typename T>
__device__ __forceinline__ bool rel_accept(T a, T m, const Consts<T>& c) {
    using F = Ty<T>;
    if (!(a <= F::mul(T(2), m) && m <= F::mul(T(2), a))) return false;
    const T d = F::fabs_(F::sub(a, m));  // exact (Sterbenz)
    const T lo = (a < m) ? a : m;
    if (lo < F::tiny()) {  // exact power-of-two rescale keeps t out of the subnormal range
        const T sc = F::rescale();
        const T t = F::mul(F::mul(lo, sc), c.chk);
        return (t >= F::nmin()) && (F::mul(d, sc) <= t);
    }
    const T t = F::mul(lo, c.chk);  // scaling by 1 is exact, so it is left out
    return (t >= F::nmin()) && (d <= t);
}

// REL: returns false for an outlier; the stored bin is 2b + signbit.
template <typename T>
__device__ __forceinline__ bool rel_quant(T x, const Consts<T>& c, int32_t& bin) {
    using F = Ty<T>;
    using U = typename F::U;
    const U u = F::bits(x);
    const U E = (u >> F::kP) & F::kExpAll;
    if (E == 0 || E == F::kExpAll) return false;  // zero, denormal, Inf, NaN
    const U sign_bit = u >> (sizeof(U) * 8 - 1);
    const T a = F::from_bits(u & ~((U)1 << (sizeof(U) * 8 - 1)));
    const T L = log2approx<T>(u);
    const T q = F::mul(L, c.inv);
    if (!(F::fabs_(q) < T(kMaxBinRel))) return false;
    int32_t b;
    T bf;
    Cv<T>::round(q, b, bf);
    if ((uint32_t)(b + (kMaxBinRel - 1)) > (uint32_t)(2 * (kMaxBinRel - 1))) return false;  // Sec. 3.3
    const T Lr = F::mul(bf, c.scale);
    const T bb = F::add(Lr, F::bias_f());
    if (!(bb >= T(1) && bb < F::top_bb())) return false;
    const T m = F::from_bits(pow2approx_bits<T>(bb));
    if (!rel_accept<T>(a, m, c)) return false;
    bin = (int32_t)(((uint32_t)b << 1) | (uint32_t)sign_bit);
    return true;
}

// REL with the math library's log2 / exp2 (ablation): the same bin rule and
// the same acceptance test, with L = log2(a) and m = exp2(b step).  m must be
// finite and normal.  The library results differ between devices and
// libraries (Sec. 2.3), so only a decoder with the same library reproduces m.
template <typename T>
__device__ __forceinline__ T lib_log2(T a) {
    if constexpr (sizeof(T) == 4) return log2f(a);
    else return log2(a);
}
template <typename T>
__device__ __forceinline__ T lib_exp2(T a) {
    if constexpr (sizeof(T) == 4) return exp2f(a);
    else return exp2(a);
}

template <typename T>
__device__ __forceinline__ bool rel_quant_lib(T x, const Consts<T>& c, int32_t& bin) {
    using F = Ty<T>;
    using U = typename F::U;
    const U u = F::bits(x);
    const U E = (u >> F::kP) & F::kExpAll;
    if (E == 0 || E == F::kExpAll) return false;  // zero, denormal, Inf, NaN
    const U sign_bit = u >> (sizeof(U) * 8 - 1);
    const T a = F::from_bits(u & ~((U)1 << (sizeof(U) * 8 - 1)));
    const T q = F::mul(lib_log2<T>(a), c.inv);
    if (!(F::fabs_(q) < T(kMaxBinRel))) return false;
    int32_t b;
    T bf;
    Cv<T>::round(q, b, bf);
    if ((uint32_t)(b + (kMaxBinRel - 1)) > (uint32_t)(2 * (kMaxBinRel - 1))) return false;  // Sec. 3.3
    const T m = lib_exp2<T>(F::mul(bf, c.scale));
    const U Em = (F::bits(m) >> F::kP) & F::kExpAll;
    if (Em == 0 || Em == F::kExpAll) return false;  // m not finite and normal
    if (!rel_accept<T>(a, m, c)) return false;
    bin = (int32_t)(((uint32_t)b << 1) | (uint32_t)sign_bit);
    return true;
}

template <typename T>
__device__ __forceinline__ T rel_recon_lib(int32_t bin, const Consts<T>& c) {
    using F = Ty<T>;
    using U = typename F::U;
    const U s = (U)(bin & 1);
    const T m = lib_exp2<T>(F::mul(Cv<T>::from_int(bin >> 1), c.scale));
    return F::from_bits(F::bits(m) | (s << (sizeof(U) * 8 - 1)));
}

// 16-bit ABS / NOA: abs_quant's float recipe on the widened value x; the
// check tests the decoder's output, the reconstruction rounded to the 16-bit
// format T.  The subtraction is exact wherever the comparison is close (the
// two values lie within a factor of about 2 of each other and have at most
// 11 significant bits, or the reconstruction is 0).
template <typename T>
__device__ __forceinline__ bool abs_quant16(float x, const Consts<float>& c, int32_t& bin) {
    using F = Ty<T>;
    const float q = __fmul_rn(x, c.inv);
    if (!(fabsf(q) < (float)kMaxBinAbs)) return false;
    int32_t b;
    float bf;
    Cv<float>::round(q, b, bf);
    if ((uint32_t)(b + (kMaxBinAbs - 1)) > (uint32_t)(2 * (kMaxBinAbs - 1))) return false;  // Sec. 3.3
    const float r = F::widen(F::narrow(__fmul_rn(bf, c.scale)));
    if (!(fabsf(__fsub_rn(x, r)) <= c.ebT)) return false;
    bin = b;
    return true;
}

// 16-bit REL: rel_quant's float recipe on the widened value, accepting the
// decoder's magnitude RN16(m) in place of m (an Inf or 0 fails the ratio
// test).  Float zeros, denormals (bfloat16 subnormals), Inf and NaN are
// outliers; binary16 subnormals are normal floats and are quantized.
template <typename T>
__device__ __forceinline__ bool rel_quant16(float x, const Consts<float>& c, int32_t& bin) {
    using F = Ty<T>;
    const uint32_t u = __float_as_uint(x);
    const uint32_t E = (u >> 23) & 0xFFu;
    if (E == 0u || E == 0xFFu) return false;
    const float a = __uint_as_float(u & 0x7FFFFFFFu);
    const float q = __fmul_rn(log2approx<float>(u), c.inv);
    if (!(fabsf(q) < (float)kMaxBinRel)) return false;
    int32_t b;
    float bf;
    Cv<float>::round(q, b, bf);
    if ((uint32_t)(b + (kMaxBinRel - 1)) > (uint32_t)(2 * (kMaxBinRel - 1))) return false;  // Sec. 3.3
    const float bb = __fadd_rn(__fmul_rn(bf, c.scale), 127.0f);
    if (!(bb >= 1.0f && bb < 255.0f)) return false;
    const float m = F::widen(F::narrow(__uint_as_float(pow2approx_bits<float>(bb))));
    if (!rel_accept<float>(a, m, c)) return false;
    bin = (int32_t)(((uint32_t)b << 1) | (u >> 31));
    return true;
}

// What the four-value fast paths below do with a float reconstruction before
// checking it: Keep32 (float32 data) leaves it; Round16<T> replaces it by the
// decoder's 16-bit value, widened back (two packed conversions per four
// values).  Each also names the per-value recipes of its data type, used
// where the fast code does not apply.
struct Keep32 {
    static __device__ __forceinline__ void apply(float v[4]) {}
    template <bool CHECK>
    static __device__ __forceinline__ bool abs1(float x, const Consts<float>& c, int32_t& bin) {
        return abs_quant<float, CHECK>(x, c, bin);
    }
    static __device__ __forceinline__ bool rel1(float x, const Consts<float>& c, int32_t& bin) {
        return rel_quant<float>(x, c, bin);
    }
};

template <typename T>
struct Round16;

template <typename T>
struct Round16Base {
    template <bool CHECK>
    static __device__ __forceinline__ bool abs1(float x, const Consts<float>& c, int32_t& bin) {
        static_assert(CHECK, "16-bit formats: the protected quantizer only");
        return abs_quant16<T>(x, c, bin);
    }
    static __device__ __forceinline__ bool rel1(float x, const Consts<float>& c, int32_t& bin) {
        return rel_quant16<T>(x, c, bin);
    }
};

template <>
struct Round16<f16s> : Round16Base<f16s> {
    static __device__ __forceinline__ void apply(float v[4]) {
        const float2 a = __half22float2(__floats2half2_rn(v[0], v[1]));
        const float2 b = __half22float2(__floats2half2_rn(v[2], v[3]));
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
};

template <>
struct Round16<bf16s> : Round16Base<bf16s> {
    static __device__ __forceinline__ void apply(float v[4]) {
        const __nv_bfloat162 a = __floats2bfloat162_rn(v[0], v[1]);
        const __nv_bfloat162 b = __floats2bfloat162_rn(v[2], v[3]);
        v[0] = __uint_as_float((uint32_t)__bfloat16_as_ushort(a.x) << 16);
        v[1] = __uint_as_float((uint32_t)__bfloat16_as_ushort(a.y) << 16);
        v[2] = __uint_as_float((uint32_t)__bfloat16_as_ushort(b.x) << 16);
        v[3] = __uint_as_float((uint32_t)__bfloat16_as_ushort(b.y) << 16);
    }
};

// ---------------------------------------------------------------------------
// Four values at a time (one 128-bit load), float32.  When every lane of the
// warp has |q| < 2^22 for all four of its values -- the usual case -- one
// warp-uniform branch selects straight-line code without per-value branches;
// otherwise (ABS) the per-value recipes above run, or (REL) the same
// straight-line code with a rounding that is exact for any |q| < 2^29.  All
// give identical results: the fast code is the same sequence of IEEE
// operations, and the checks it leaves out are implied (|q| < 2^22: no
// integer overflow, |b| <= 2^22 < maxbin; the REL implications are listed at
// rel_fast4_f32).  Returns the 4-bit outlier nibble; bins of outliers are 0.
// ---------------------------------------------------------------------------
template <bool CHECK = true, typename R = Keep32>
__device__ __forceinline__ uint32_t abs_quant4_f32(const float x[4], const Consts<float>& c, int32_t b[4]) {
    float q[4];
    bool small = true;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        q[k] = __fmul_rn(x[k], c.inv);
        small &= fabsf(q[k]) < 0x1p22f;
    }
    uint32_t nb = 0;
    if (__all_sync(0xFFFFFFFFu, small)) {
        int32_t bi[4];
        float recon[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const float t = __fadd_rn(q[k], 0x1.8p23f);
            bi[k] = __float_as_int(t) - 0x4B400000;
            recon[k] = __fmul_rn(__fsub_rn(t, 0x1.8p23f), c.scale);
        }
        if constexpr (CHECK) R::apply(recon);
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const bool ok = !CHECK || fabsf(__fsub_rn(x[k], recon[k])) <= c.ebT;
            b[k] = ok ? bi[k] : 0;
            nb |= ok ? 0u : (1u << k);
        }
    } else {
#pragma unroll
        for (int k = 0; k < 4; k++) {
            int32_t bin = 0;
            const bool ok = R::template abs1<CHECK>(x[k], c, bin);
            b[k] = ok ? bin : 0;
            nb |= ok ? 0u : (1u << k);
        }
    }
    return nb;
}

// The fast REL code for four values whose |q| < 2^22 (see rel_quant4_f32).
// It computes exactly what rel_quant<float> computes, with fewer instructions:
//  * pow2approx(bb) for 1 <= bb < 255: with k = floor(bb) and frac = bb - k,
//    its bit pattern (k << 23) | frac 2^23 is the integer bb 2^23 (frac is a
//    multiple of 2^-23 because bb >= 1), so one exact scaling by 2^23 and one
//    exact conversion give it;
//  * 1 <= bb < 255 is one unsigned comparison of bit patterns (bit patterns of
//    non-negative floats are ordered like the floats; negative ones are huge);
//  * RATIO = false leaves out the test m/2 <= a <= 2m, which the acceptance
//    test implies when chk <= 1/2: if it fails, |a - m| > lo exactly, so
//    d = RN(|a - m|) >= lo (lo is a float), while t = RN(lo chk) <= RN(lo / 2)
//    < lo (the same holds after the exact rescale), so d <= t fails too;
//  * WIDE = false (every |q| of the warp below 2^22) rounds with the
//    1.5 2^23 addition; WIDE = true rounds with rintf / __float2int_rn, exact
//    for every |q| < 2^29 (a float of magnitude >= 2^23 is an integer), and
//    makes |q| >= 2^29 an outlier: that is the range test, and the two-sided
//    bin test then holds because rint(q) < 2^29 for q < 2^29;
//  * the exact rescale for tiny values runs only in warps that have one, and
//    with RATIO = false "tiny" means lo < T = 2^(1 - e_c) (e_c = the biased
//    exponent of chk <= 1/2, so T >= FLT_MIN / chk and T >= 2^-125) rather
//    than the recipe's 2^-62: for T <= lo < 2^-62 the rescale is exact both
//    ways (lo chk >= FLT_MIN, so RN(lo 2^64 chk) = RN(lo chk) 2^64 and
//    d 2^64 <= t <=> d <= RN(lo chk)), so skipping it changes nothing;
//  * a warp whose only tiny values are zeros and denormals (a < FLT_MIN, all
//    outliers) or NaN still takes the straight-line code, which rejects them
//    without a test of their own: RN(lo chk) <= RN(a / 2) < FLT_MIN for
//    a < FLT_MIN, and d is NaN for a NaN a;
//  * in a warp without tiny values (every lo = min(a, m) >= T, apart from
//    the rejected a < FLT_MIN) and with RATIO = false, the special-value and
//    bb-range tests are implied as well: a zero or denormal a is rejected
//    explicitly or makes lo tiny; bb < 1 (m = bb 2^23 converted is then below
//    2^-126 < T, or 0 for bb < 0) makes lo tiny; an Inf or NaN a makes d Inf
//    or NaN; bb >= 255 makes m +Inf, a NaN, or a negative value (bit 31 set:
//    then t = RN(lo chk) <= 0 < FLT_MIN); each of these fails d <= t or
//    t >= FLT_MIN.
template <bool RATIO, bool WIDE, typename R = Keep32>
__device__ __forceinline__ uint32_t rel_fast4_f32(const float x[4], const float q[4], const Consts<float>& c,
                                                  int32_t b[4]) {
    float a[4], m[4], lo[4], bb[4];
    int32_t bin[4];
    bool inr[4];
    bool tiny = false;
    // tiny threshold: 2^(1 - e_c) for chk <= 1/2 (see above), else the recipe's 2^-62
    const float T = RATIO ? 0x1p-62f : __uint_as_float((128u - ((__float_as_uint(c.chk) >> 23) & 0xFFu)) << 23);
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const uint32_t u = __float_as_uint(x[k]);
        a[k] = __uint_as_float(u & 0x7FFFFFFFu);
        float bf;
        int32_t bi;
        if (WIDE) {
            bf = rintf(q[k]);
            bi = __float2int_rn(q[k]);
            inr[k] = fabsf(q[k]) < 0x1p29f;
        } else {
            const float t = __fadd_rn(q[k], 0x1.8p23f);
            bi = __float_as_int(t) - 0x4B400000;
            bf = __fsub_rn(t, 0x1.8p23f);
            inr[k] = true;
        }
        bin[k] = (int32_t)(((uint32_t)bi << 1) | (u >> 31));
        const float Lr = __fmul_rn(bf, c.scale);
        bb[k] = __fadd_rn(Lr, 127.0f);
        m[k] = __uint_as_float(__float2uint_rz(__fmul_rn(bb[k], 0x1p23f)));
    }
    R::apply(m);  // the decoder's magnitudes
#pragma unroll
    for (int k = 0; k < 4; k++) {
        lo[k] = fminf(a[k], m[k]);
        tiny |= lo[k] < T;
    }
    uint32_t nb = 0;
    if (!RATIO) {
        // Straight-line code unless a tiny value other than a zero, a
        // denormal or NaN needs the rescale.  A zero or denormal a (a <
        // FLT_MIN) is rejected there without a test of its own: lo <= a and
        // chk <= 1/2 give RN(lo chk) <= FLT_MIN / 2 < FLT_MIN; a NaN a makes
        // d NaN.
        bool fast = !__any_sync(0xFFFFFFFFu, tiny);
        if (!fast) {
            bool tiny2 = false;
#pragma unroll
            for (int k = 0; k < 4; k++) tiny2 |= lo[k] < T && a[k] >= FLT_MIN;
            fast = !__any_sync(0xFFFFFFFFu, tiny2);
        }
        if (fast) {
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const float d = fabsf(__fsub_rn(a[k], m[k]));  // exact (Sterbenz) when accepted
                const float tt = __fmul_rn(lo[k], c.chk);
                const bool ok = inr[k] && (tt >= FLT_MIN) && (d <= tt);
                b[k] = ok ? bin[k] : 0;
                nb |= ok ? 0u : (1u << k);
            }
            return nb;
        }
    }
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const uint32_t E = (__float_as_uint(x[k]) >> 23) & 0xFFu;
        bool ok = inr[k] && (E - 1u < 254u) &&
                  (__float_as_uint(bb[k]) - 0x3F800000u < 0x437F0000u - 0x3F800000u);
        if (RATIO) ok = ok && (a[k] <= __fmul_rn(2.0f, m[k])) && (m[k] <= __fmul_rn(2.0f, a[k]));
        const float d = fabsf(__fsub_rn(a[k], m[k]));
        // exact power-of-two rescale of tiny values; a scale of 1 is exact too,
        // so selecting the factor gives both branches of rel_quant at once
        const float sc = lo[k] < 0x1p-62f ? 0x1p64f : 1.0f;
        const float tt = __fmul_rn(__fmul_rn(lo[k], sc), c.chk);
        ok = ok && (tt >= FLT_MIN) && (__fmul_rn(d, sc) <= tt);
        b[k] = ok ? bin[k] : 0;
        nb |= ok ? 0u : (1u << k);
    }
    return nb;
}

template <typename R = Keep32>
__device__ __forceinline__ uint32_t rel_quant4_f32(const float x[4], const Consts<float>& c, int32_t b[4]) {
    float q[4];
    bool small = true;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const float L = log2approx<float>(__float_as_uint(x[k]));  // finite for every bit pattern
        q[k] = __fmul_rn(L, c.inv);
        small &= fabsf(q[k]) < 0x1p22f;
    }
    const bool narrow = __all_sync(0xFFFFFFFFu, small);
    if (c.chk <= 0.5f)
        return narrow ? rel_fast4_f32<false, false, R>(x, q, c, b) : rel_fast4_f32<false, true, R>(x, q, c, b);
    return narrow ? rel_fast4_f32<true, false, R>(x, q, c, b) : rel_fast4_f32<true, true, R>(x, q, c, b);
}

// ---------------------------------------------------------------------------
// float64 with few FP64 operations.  The FP64 pipe of this GPU issues only
// about 1.6 multiplications per clock per SM, so the float64 recipes keep on
// it one multiplication per value (q; REL also log2approx's addition), run
// the double-check there only where its outcome is not already certain (see
// abs_quant_f64, rel_quant_f64), and do the rest exactly on the bit patterns
// with integer operations:
//   * |v| < 2^w and |a| <= |b| as integer comparisons of the (sign-cleared)
//     bit patterns: for non-negative IEEE doubles, including +Inf and NaN
//     patterns, numeric order is the order of the bits;
//   * rint of a double with |q| < 2^30 from its fields, round half to even;
//   * an integer below 2^53 converted to the double with its exact value;
//   * pow2approx of bb in [1, 2047): floor and fraction read off bb's fields;
//   * the exact difference of two positive doubles within a factor 2 of each
//     other (an integer subtraction of aligned significands, always exact).
// Every helper returns exactly what the double operation(s) it replaces
// return; the float64 parity tests run both against the oracle.
// ---------------------------------------------------------------------------
constexpr uint64_t kD_MANT = 0x000FFFFFFFFFFFFFull;
constexpr uint64_t kD_SIGN = 0x8000000000000000ull;

__device__ __forceinline__ uint64_t dbits(double v) { return (uint64_t)__double_as_longlong(v); }
__device__ __forceinline__ double dfrom(uint64_t u) { return __longlong_as_double((long long)u); }

// The bits of |v| from the bits u of v: the sign bit cleared by an integer
// instruction.  Written as inline PTX because the compiler otherwise turns
// the mask of a double's bit pattern into a floating-point absolute value,
// which this GPU executes on its FP64 pipe.
__device__ __forceinline__ uint64_t clear_sign(uint64_t u) {
    uint64_t r;
    asm("and.b64 %0, %1, 0x7FFFFFFFFFFFFFFF;" : "=l"(r) : "l"(u));
    return r;
}

// rint(q) for a double q with |q| < 2^30 (caller checks), round half to even.
__device__ __forceinline__ int32_t rint_d_small(uint64_t u) {
    const int e = (int)((u >> 52) & 0x7FF);
    const int sh = 1075 - e;  // q = m 2^-sh, m = 1.M 2^52
    if (sh > 53) return 0;    // |q| < 1/2 (or zero / denormal)
    const uint64_t m = (u & kD_MANT) | (1ull << 52);
    const uint64_t ip = m >> sh;
    const uint64_t rem = m & ((1ull << sh) - 1);
    const uint64_t half = 1ull << (sh - 1);
    const uint64_t r = ip + ((rem > half || (rem == half && (ip & 1))) ? 1 : 0);
    return (u & kD_SIGN) ? -(int32_t)r : (int32_t)r;
}

// The integer part and the top 32 bits of the fraction of a double q with
// |q| < 2^30 (caller checks), by two funnel shifts of its significand: q =
// ip + f 2^-32 + delta, 0 <= delta < 2^-32 (sign apart).  For |q| < 1/2 it
// returns ip = 0, f = 0 and sets small.
__device__ __forceinline__ uint32_t d_int_frac(uint64_t u, uint32_t& f, bool& small) {
    const uint32_t hi = (uint32_t)(u >> 32);
    const int sh = 1075 - (int)((hi >> 20) & 0x7FFu);  // q = m 2^-sh, 23 <= sh when |q| < 2^30
    small = sh > 53;
    if (small) {
        f = 0;
        return 0;
    }
    const uint64_t m = (u & kD_MANT) | (1ull << 52);
    f = (uint32_t)((m << (64 - sh)) >> 32);
    return (uint32_t)(m >> sh);
}

// rint(q), round half to even, for |q| < 2^30 (caller checks): the fraction's
// top 32 bits decide unless they are exactly 1/2, where rint_d_small does.
__device__ __forceinline__ int32_t rint_d_fast(uint64_t u) {
    uint32_t f;
    bool small;
    const uint32_t ip = d_int_frac(u, f, small);
    if (small) return 0;  // |q| < 1/2
    if (f == 0x80000000u) return rint_d_small(u);
    const uint32_t r = ip + (f > 0x80000000u ? 1u : 0u);
    return (u & kD_SIGN) ? -(int32_t)r : (int32_t)r;
}

// rint(q) as rint_d_fast, and whether q lies at least 2^-20 away from the
// midpoint between two integers (clear).  With q = ip + F 2^-32 + delta:
// |F - 2^31| > 2^12 gives |frac - 1/2| >= 2^-20 + 2^-32 - delta > 2^-20 and
// fixes the rounding direction; |q| <= 1/2 - 2^-20 is clear as well (its
// high word below that of 0x3FDFFFFC00000000, a conservative test).  Where
// clear is false the returned bin is exact but the caller checks anyway.
__device__ __forceinline__ int32_t rint_d_fast_clear(uint64_t u, bool& clear) {
    uint32_t f;
    bool small;
    const uint32_t ip = d_int_frac(u, f, small);
    if (small) {
        clear = ((uint32_t)(u >> 32) & 0x7FFFFFFFu) < 0x3FDFFFFCu;
        return 0;
    }
    const uint32_t d = f > 0x80000000u ? f - 0x80000000u : 0x80000000u - f;
    clear = d > 0x1000u;
    if (!clear) return rint_d_small(u);
    const uint32_t r = ip + (f > 0x80000000u ? 1u : 0u);
    return (u & kD_SIGN) ? -(int32_t)r : (int32_t)r;
}

// The double with the exact value of integer i, |i| < 2^20 (32-bit work).
__device__ __forceinline__ uint64_t small_int_to_dbits(int32_t i) {
    if (i == 0) return 0;
    const uint32_t a = (uint32_t)(i < 0 ? -i : i);
    const int top = 31 - __clz((int)a);
    const uint32_t hi = ((uint32_t)(top + 1023) << 20) | ((a << (20 - top)) & 0xFFFFFu);
    return ((uint64_t)(hi | (i < 0 ? 0x80000000u : 0u)) << 32);
}

// The double with the exact value of integer i, |i| < 2^53.
__device__ __forceinline__ uint64_t int_to_dbits(int64_t i) {
    if (i == 0) return 0;
    const uint64_t sgn = i < 0 ? kD_SIGN : 0;
    const uint64_t a = (uint64_t)(i < 0 ? -i : i);
    const int top = 63 - __clzll((long long)a);
    return sgn | ((uint64_t)(top + 1023) << 52) | ((a << (52 - top)) & kD_MANT);
}

// pow2approx bits of bb in [1, 2047) (caller checks): 2^(k-1023)(1 + bb - k).
__device__ __forceinline__ uint64_t pow2approx_dbits(uint64_t ub) {
    int e = (int)((ub >> 52) & 0x7FF) - 1023;  // 0..10 for a valid bb
    e = e < 0 ? 0 : (e > 10 ? 10 : e);          // garbage in, garbage out, no undefined shift
    const uint64_t m = ub & kD_MANT;
    const uint64_t k = (1ull << e) + (m >> (52 - e));
    return (k << 52) | ((m << e) & kD_MANT);
}

// Exact |a - b| for positive normal doubles with a/2 <= b <= 2a; returns bits.
__device__ __forceinline__ uint64_t absdiff_close_dbits(uint64_t ua, uint64_t ub) {
    if (ua < ub) { const uint64_t t = ua; ua = ub; ub = t; }  // ua >= ub
    const int ea = (int)(ua >> 52), eb = (int)(ub >> 52);     // eb = ea or ea - 1
    const uint64_t ma = (ua & kD_MANT) | (1ull << 52), mb = (ub & kD_MANT) | (1ull << 52);
    const uint64_t D = (ma << (ea - eb)) - mb;                // in units of 2^(eb - 1075)
    if (D == 0) return 0;
    const int top = 63 - __clzll((long long)D);               // D < 2^54; the result is exact
    const int e = eb + top - 52;                              // biased exponent of the difference
    if (e >= 1) return ((uint64_t)e << 52) | ((D << (52 - top)) & kD_MANT);
    return D << (eb - 1 > 0 ? eb - 1 : 0);                   // subnormal result: units of 2^-1074
}

// The double-check of Sec. 3.1 for float64 ABS / NOA, on the FP64 pipe:
// |RN(x - RN(b eb2))| <= eb_T.  Out of line: only values that lie within
// 2^-20 of a bin edge run it (see abs_quant_f64).
static __device__ __noinline__ bool abs_check_f64(double x, int32_t b, double eb2, double ebT) {
    const double recon = __dmul_rn(dfrom(int_to_dbits(b)), eb2);
    return clear_sign(dbits(__dsub_rn(x, recon))) <= dbits(ebT);
}

// ABS / NOA on float64.  q = RN(x inv) and b = rint(q) as always; the
// double-check then runs only where its outcome is not already certain.
// With e = eb2 = 2 eb_T (exact), inv = (1/e)(1 + d1), q = x inv (1 + d2)
// and recon = b e (1 + d3), |di| <= u = 2^-53 (q is normal when b != 0; when
// q is subnormal, b = 0 and |x| < 2^-1022 e (1 + u) is far below eb_T):
//   x - b e = e (q / ((1 + d1)(1 + d2)) - b),  so
//   |x - recon| <= e (|q - b| + 2.0001 u |q| + u |b|)
//              <= e (|q - b| + 3.0001 u |q| + u / 2)      (|b| <= |q| + 1/2)
//              <  e (|q - b| + 2^-20)                    (|q| < 2^30).
// So |q - b| <= 1/2 - 2^-20 gives |x - recon| <= e / 2 = eb_T exactly, and
// then RN(|x - recon|) <= eb_T as well (eb_T is a double): the check passes.
// recon must not overflow for this (d3 above): with |x| < 2^1022 and b != 0,
// |q| >= 1/2 gives e < 2^1023 and |b e| < |x| (1 + 2u) + e / 2 < DBL_MAX.
// Every other value (a fraction of about 2^-19 of smooth data, and any
// |x| >= 2^1022) runs the check.
template <bool CHECK = true>
__device__ __forceinline__ bool abs_quant_f64(double x, const Consts<double>& c, int32_t& bin) {
    const double q = __dmul_rn(x, c.inv);
    const uint64_t uq = clear_sign(dbits(q));
    if (!(uq < 0x41D0000000000000ull)) return false;  // !(|q| < 2^30): also NaN
    bool clear;
    const int32_t b = rint_d_fast_clear(dbits(q), clear);
    if ((uint32_t)(b + (kMaxBinAbs - 1)) > (uint32_t)(2 * (kMaxBinAbs - 1))) return false;  // Sec. 3.3
    if constexpr (CHECK) {
        clear = clear && ((uint32_t)(dbits(x) >> 32) & 0x7FFFFFFFu) < 0x7FD00000u;  // |x| < 2^1022
        if (!clear && !abs_check_f64(x, b, c.scale, c.ebT)) return false;
    }
    bin = b;
    return true;
}

// The rest of the float64 REL recipe after the bin b: m = pow2approx(RN(RN(b
// step) + 1023)), the range test of bb, m/2 <= a <= 2m, and |a - m| <=
// RN(min(a, m) chk) with that product normal (exact rescale below 2^-511).
// Out of line: rel_quant_f64 calls it only where the outcome is not certain.
static __device__ __noinline__ bool rel_check_f64(uint64_t u, int32_t b, double step, double chk) {
    const uint64_t ua = clear_sign(u);
    const double Lr = __dmul_rn(dfrom(int_to_dbits(b)), step);
    const double bb = __dadd_rn(Lr, 1023.0);
    const uint64_t ubb = dbits(bb);
    if (!(ubb >= 0x3FF0000000000000ull && ubb < 0x409FFC0000000000ull)) return false;  // 1 <= bb < 2047
    const uint64_t um = pow2approx_dbits(ubb);
    // m/2 <= a <= 2m: doubling adds one to the exponent field (an overflow gives +Inf's bits)
    if (!(ua <= um + (1ull << 52) && um <= ua + (1ull << 52))) return false;
    const uint64_t ud = absdiff_close_dbits(ua, um);
    const uint64_t ulo = ua < um ? ua : um;
    if (ulo < 0x2000000000000000ull) {  // lo < 2^-511: exact rescale by 2^512 (rare)
        const double sc = 0x1p512;
        const double t = __dmul_rn(__dmul_rn(dfrom(ulo), sc), chk);
        return (t >= DBL_MIN) && (__dmul_rn(dfrom(ud), sc) <= t);
    }
    const uint64_t ut = dbits(__dmul_rn(dfrom(ulo), chk));
    return (ut >= 0x0010000000000000ull) && (ud <= ut);  // t normal, d <= t
}

// REL on float64.  q = RN(L inv), L = log2approx(a), and b = rint(q) as
// always; the rest of the check runs only where its outcome is not certain.
// With a = 2^(E-1023) (1 + f), f = M 2^-52, log2approx's exact value plus
// 1023 is E + f.  Each later rounding moves the log-domain value by at most:
// L: 2^-44; q: |L| 2.0001 u <= 2^-42 (u = 2^-53, |L| < 1024); Lr = RN(b step):
// 2^-43; bb = RN(Lr + 1023): 2^-43.  So bb = E + f + (b - q) step + eps with
// |eps| < 2^-40 and |b - q| <= 1/2.  If f lies at least step/2 + 2^-40 inside
// its binade (cert_w <= M < 2^52 - cert_w, cert_w = ceil((step/2 + 2^-40)
// 2^52)), floor(bb) = E: bb is in range, m = 2^(E-1023) (1 + frac(bb)) is in
// a's binade (so m/2 <= a <= 2m and a - m is exact) and
// |a - m| <= 2^(E-1023) (step/2 + 2^-40).  The host sets cert_w only if
// chk - step/2 >= 2^-39, so that this is at most 2^(E-1023) chk (1 - u) <=
// RN(min(a, m) chk) = t; cert_emin = max(512, 1027 - exponent field of chk)
// keeps min(a, m) >= 2^-511 (no rescale) and t normal.  The acceptance test
// then passes.
__device__ __forceinline__ bool rel_quant_f64(double x, const Consts<double>& c, int32_t& bin) {
    const uint64_t u = dbits(x);
    const uint64_t E = (u >> 52) & 0x7FF;
    if (E == 0 || E == 0x7FF) return false;  // zero, denormal, Inf, NaN
    // log2approx (Sec. 3.2): 1.M + (E - 1024), one FP64 addition (the FP64 pipe
    // has room here; rounding the exact fixed-point sum with integers costs ~28
    // instructions)
    const double L = __dadd_rn(dfrom(0x3FF0000000000000ull | (u & kD_MANT)), dfrom(small_int_to_dbits((int32_t)E - 1024)));
    const double q = __dmul_rn(L, c.inv);
    const uint64_t uq = clear_sign(dbits(q));
    if (!(uq < 0x41C0000000000000ull)) return false;  // !(|q| < 2^29)
    const int32_t b = rint_d_fast(dbits(q));
    if ((uint32_t)(b + (kMaxBinRel - 1)) > (uint32_t)(2 * (kMaxBinRel - 1))) return false;  // Sec. 3.3
    const uint64_t M = u & kD_MANT;
    const bool sure = c.cert_w != 0 && E >= c.cert_emin && M >= c.cert_w && M < (1ull << 52) - c.cert_w;
    if (!sure && !rel_check_f64(u, b, c.scale, c.chk)) return false;
    bin = (int32_t)(((uint32_t)b << 1) | (uint32_t)(u >> 63));
    return true;
}

__device__ __forceinline__ double abs_recon_f64(int32_t bin, const Consts<double>& c) {
    return __dmul_rn(dfrom(int_to_dbits(bin)), c.scale);
}

__device__ __forceinline__ double rel_recon_f64(int32_t bin, const Consts<double>& c) {
    const int32_t b = bin >> 1;
    const double bb = __dadd_rn(__dmul_rn(dfrom(int_to_dbits(b)), c.scale), 1023.0);
    return dfrom(pow2approx_dbits(dbits(bb)) | ((uint64_t)(bin & 1) << 63));
}

// One value: the float32 recipes above, the float64 ones with few FP64 ops,
// or the 16-bit ones.
template <typename T, int MODE>
__device__ __forceinline__ bool quant1(T x, const Consts<CT<T>>& c, int32_t& bin) {
    if constexpr (is16<T>()) {
        static_assert(MODE == LCQ_ABS || MODE == LCQ_REL, "16-bit formats: ABS/NOA and REL only");
        if constexpr (MODE == LCQ_REL) return rel_quant16<T>(Ty<T>::widen(x), c, bin);
        else return abs_quant16<T>(Ty<T>::widen(x), c, bin);
    } else if constexpr (MODE == kModeRelLib) {
        return rel_quant_lib<T>(x, c, bin);
    } else if constexpr (sizeof(T) == 8) {
        if constexpr (MODE == LCQ_REL) return rel_quant_f64(x, c, bin);
        else return abs_quant_f64<MODE != kModeAbsNoCheck>(x, c, bin);
    } else {
        if constexpr (MODE == LCQ_REL) return rel_quant<T>(x, c, bin);
        else return abs_quant<T, MODE != kModeAbsNoCheck>(x, c, bin);
    }
}

template <typename T, int MODE>
__device__ __forceinline__ uint32_t quant4(const T x[4], const Consts<CT<T>>& c, int32_t b[4]) {
    if constexpr (is16<T>()) {
        float xf[4];
        Ty<T>::widen4(x, xf);
        if constexpr (MODE == LCQ_REL) return rel_quant4_f32<Round16<T>>(xf, c, b);
        else return abs_quant4_f32<true, Round16<T>>(xf, c, b);
    } else if constexpr (sizeof(T) == 4 && MODE == LCQ_REL) {
        return rel_quant4_f32(x, c, b);
    } else if constexpr (sizeof(T) == 4 && MODE != kModeRelLib) {
        return abs_quant4_f32<MODE != kModeAbsNoCheck>(x, c, b);
    } else {
        uint32_t nb = 0;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            int32_t bin = 0;
            const bool ok = quant1<T, MODE>(x[k], c, bin);
            b[k] = ok ? bin : 0;
            nb |= ok ? 0u : (1u << k);
        }
        return nb;
    }
}

template <typename T>
__device__ __forceinline__ T rel_recon(int32_t bin, const Consts<T>& c) {
    using F = Ty<T>;
    using U = typename F::U;
    const U s = (U)(bin & 1);
    const int32_t b = bin >> 1;  // arithmetic shift: (bin - s) / 2
    const T Lr = F::mul(Cv<T>::from_int(b), c.scale);
    const T bb = F::add(Lr, F::bias_f());
    return F::from_bits(pow2approx_bits<T>(bb) | (s << (sizeof(U) * 8 - 1)));
}

// Reconstruction of one value, as the decoder computes it.
template <typename T>
__device__ __forceinline__ T recon1(bool rel, int32_t bin, const Consts<T>& c) {
    if constexpr (sizeof(T) == 8) return rel ? rel_recon_f64(bin, c) : abs_recon_f64(bin, c);
    else return rel ? rel_recon<T>(bin, c) : abs_recon<T>(bin, c);
}

// The decoder's output value: recon1, rounded to the 16-bit format for the
// 16-bit formats.
template <typename T>
__device__ __forceinline__ T recon_out(bool rel, int32_t bin, const Consts<CT<T>>& c) {
    if constexpr (is16<T>()) return Ty<T>::narrow(recon1<float>(rel, bin, c));
    else return recon1<T>(rel, bin, c);
}

// ---------------------------------------------------------------------------
// Workspace head and launch bookkeeping
// ---------------------------------------------------------------------------

// The 256-byte head of every workspace (what follows it is laid out by each
// entry point).
struct WsHead {
    uint32_t ticket;  // next scan tile index (handed out dynamically)
    uint32_t done;    // CTAs finished; the last one resets ticket/done
    uint32_t epoch;   // launch counter
    uint32_t err;     // LCQ_STATUS_* bits gathered during one launch
    uint64_t carry;   // running outlier count across chunks (decoder)
    uint32_t cdone;   // compaction CTAs finished; the last one resets it
};

// Programmatic dependent launch (PTX griddepcontrol, sm_90 and later).  A
// kernel launched with the programmatic stream serialisation attribute may
// be scheduled while the kernel before it in the stream is still running:
// pdl_wait() blocks until that kernel has completed and its memory writes
// are visible (for a plain launch it returns at once), and pdl_trigger()
// lets the next kernel be scheduled before this one ends.  Every kernel of
// the single-array path calls pdl_wait() before it touches global memory,
// so the overlap only hides launch latency.  The quantize kernel triggers
// when a CTA has finished its tiles, not at its start: CTAs of the
// compaction that were let in early made outlier-heavy calls 9% slower.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

constexpr size_t kWsHeadBytes = 256;
constexpr int kMinmaxMaxBlocks = 1184;  // 8 x 148
constexpr size_t kMinmaxPartialBytes = (size_t)kMinmaxMaxBlocks * 2 * sizeof(uint64_t);

__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t* p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u64(uint64_t* p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Test hook of the bounded waits (lcq_debug_set_scan): in a quantize launch
// the scan warp never hands scan tile drop_tile back to its compute warps,
// whose wait for it gives up after spin_limit polls with LCQ_STATUS_TIMEOUT.
struct ScanCfg {
    uint32_t spin_limit;
    uint64_t drop_tile;  // UINT64_MAX: none
};

// End-of-launch bookkeeping, called by thread 0 of every CTA after its last
// global write: the last CTA to finish hands the gathered error bits to
// *status_out (assigning on the first chunk of a call, OR-ing later) and
// resets the ticket for the next launch on this workspace.  Returns true in
// the last CTA.
__device__ __forceinline__ bool finish_launch(WsHead* ws, uint32_t epoch, uint32_t* status_out,
                                              bool assign) {
    __threadfence();
    const uint32_t prev = atomicAdd(&ws->done, 1u);
    const bool last = prev == gridDim.x - 1;
    if (last) {
        __threadfence();
        const uint32_t e = atomicExch(&ws->err, 0u);
        if (status_out) {
            if (assign) *status_out = e;
            else atomicOr(status_out, e);
        }
        atomicExch(&ws->ticket, 0u);
        atomicExch(&ws->done, 0u);
        atomicExch(&ws->epoch, epoch + 1u);
        __threadfence();
    }
    return last;
}

}  // namespace lcq
