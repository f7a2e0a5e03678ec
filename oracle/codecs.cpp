/*
 * CPU ORACLE -- TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU baseline).
 *
 * Storage-format codecs of arXiv 2112.08926, Sec. 3, written in the VALUE
 * domain: every decoder maps a code to the real number the format defines
 * (Sec. 3.1.1 floating-point form, Sec. 3.2.1 posit form, Table 2, Fig. 2), and
 * every encoder first decides which representable value the input rounds to
 * (a rule on real numbers) and then looks that value up.  No bit tricks.
 *
 * The rounding rules are the behaviour of the paper's conversion routines
 * (appendix, "Ultrafast conversion algorithms"), restated as rules on values:
 *
 *   FP16, FP16S   IEEE-754 binary16 round-to-nearest-even (Sec. 3.1.3, the
 *                 hardware conversion); FP16S scales by 2^15 in FP32 before
 *                 encoding and by 2^-15 after decoding.
 *   FP16C         1|4|11 bits, bias 15, no Inf/NaN (Sec. 3.1.2, 3.1.4):
 *                 round to nearest with ties away from zero (the rounding
 *                 increment is added to the magnitude, so halfway cases go
 *                 up in magnitude; the comment in the paper calls it
 *                 "round-to-nearest-even", the arithmetic is half-up),
 *                 subnormals kept, saturation at 1.999512.
 *   P16_0, P16_1  sign-magnitude posits with 0 / 1 exponent bits (Sec. 3.2.2,
 *                 3.2.3); the S variants scale by 2^7 before encoding and by
 *                 2^-7 after decoding.  Nearest value, ties away from zero,
 *                 with the low- and high-end rules listed at each encoder.
 *   P16_2C        asymmetric posit with 2 exponent bits covering only the
 *                 lower flank (Sec. 3.2.2), unscaled.
 *
 * Readings of the paper taken here:
 *   - codes whose 15 magnitude bits are all zero decode to +-0 for every
 *     posit format (the printed P16_0/P16_1 decoders would return
 *     -2^113 / -2^-30 for them, which no working simulation can have used);
 *   - where fewer exponent bits fit below the regime than the format has,
 *     the missing exponent bits read as zero; for P16_2C this includes the
 *     single bit that does fit when 13 regime zeros are present;
 *   - NaN inputs: see fp16c_from_float; posit encoders saturate a NaN with
 *     the sign of the input.
 *
 * Pins (tests/test_oracle_codecs.py): the posit encoders equal the rounding
 * of the exact posit bit string (Sec. 3.2.1 representation, half up on the
 * first bit cut off) over the whole FP32 range, end rules included, except
 * P16_2C below 2^-52: there the printed routine rounds the lowest numbers up
 * with increments of its own, which this file follows as value rules; that
 * sub-range is parity unpinned (its only check restates those rules).
 */
#include "oracle.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

namespace {

inline uint32_t fbits(float x) { uint32_t u; std::memcpy(&u, &x, 4); return u; }

/* floor(log2(a)) for finite a > 0 */
inline int ilog2(double a) { int e; std::frexp(a, &e); return e - 1; }

/* a rounded to a multiple of 2^(E-nf), halfway cases away from zero; a >= 0.
 * a has at most 24 significant bits, so every step is exact in double. */
inline double round_half_up_binade(double a, int E, int nf) {
    return std::ldexp(std::floor(std::ldexp(a, nf - E) + 0.5), E - nf);
}

/* ---------------- IEEE binary16 ------------------------------------------ */

double fp16_value(uint16_t c) {
    const int s = c >> 15, E = (c >> 10) & 31, M = c & 1023;
    double v;
    if (E == 31) v = M ? NAN : INFINITY;
    else if (E == 0) v = std::ldexp((double)M, -24);           /* subnormal */
    else v = std::ldexp((double)(1024 + M), E - 25);           /* 2^(E-15)(1+M/1024) */
    return s ? -v : v;
}

uint16_t fp16_from_float(float x) {
    const uint16_t s = (uint16_t)((fbits(x) >> 16) & 0x8000u);
    if (std::isnan(x)) return (uint16_t)(s | 0x7E00u);          /* a NaN; compared by class */
    const double a = std::fabs((double)x);
    /* 65520 is halfway between 65504 and 2^16; ties-to-even rounds it up: overflow */
    if (a >= 65520.0) return (uint16_t)(s | 0x7C00u);
    if (a < 0x1p-14) {                                          /* multiples of 2^-24 */
        const double n = std::nearbyint(a * 0x1p24);            /* n == 1024: smallest normal */
        return (uint16_t)(s | (uint16_t)n);
    }
    int E = ilog2(a);
    double n = std::nearbyint(std::ldexp(a, 10 - E));           /* 1024 .. 2048 */
    if (n == 2048.0) { E += 1; n = 1024.0; }
    return (uint16_t)(s | (uint16_t)(((E + 15) << 10) | ((int)n - 1024)));
}

/* ---------------- FP16C: 1 | 4 | 11, bias 15 ------------------------------ */

double fp16c_value(uint16_t c) {
    const int s = c >> 15, E = (c >> 11) & 15, M = c & 2047;
    const double v = (E == 0) ? std::ldexp((double)M, -25)            /* M * 2^-14 / 2^11 */
                              : std::ldexp((double)(2048 + M), E - 26); /* 2^(E-15)(1+M/2^11) */
    return s ? -v : v;
}

uint16_t fp16c_from_float(float x) {
    const uint32_t b = fbits(x);
    if (std::isnan(x)) {
        /* The conversion adds the rounding increment 2^11 to the raw 32-bit
         * pattern.  For the 2048 highest NaN patterns of either sign that
         * addition carries through the sign bit, leaving a zero of the
         * opposite sign; every other NaN saturates with its own sign. */
        if ((b & 0x7FFFFFFFu) >= 0x7FFFF800u) return (b & 0x80000000u) ? 0x0000 : 0x8000;
        return (uint16_t)(((b >> 16) & 0x8000u) | 0x7FFFu);
    }
    const uint16_t s = (uint16_t)((b >> 16) & 0x8000u);
    const double a = std::fabs((double)x);
    if (std::isinf(a)) return (uint16_t)(s | 0x7FFFu);
    if (a < 0x1p-14) {
        /* subnormal codes are multiples of 2^-25; 2048 * 2^-25 = 2^-14 has the
         * same pattern (0x0800) as the smallest normal number */
        return (uint16_t)(s | (uint16_t)std::floor(a * 0x1p25 + 0.5));
    }
    int E = ilog2(a);
    double n = std::floor(std::ldexp(a, 11 - E) + 0.5);         /* 2048 .. 4096 */
    if (n == 4096.0) { E += 1; n = 2048.0; }
    if (E >= 1) return (uint16_t)(s | 0x7FFFu);                 /* saturate at 1.999512 */
    return (uint16_t)(s | (uint16_t)(((E + 15) << 11) | ((int)n - 2048)));
}

/* ---------------- sign-magnitude posits ---------------------------------- */

/* Value of a symmetric sign-magnitude posit with `es` exponent bits.
 * Regime: a run of equal bits starting below the sign, ended by the opposite
 * bit (or by the end of the word); k = run-1 for a run of ones, -run for a
 * run of zeros.  Value 2^(k*2^es + e) * (1 + fraction). */
double posit_sm_value(uint16_t c, int es) {
    const int s = c >> 15;
    const uint32_t mag = c & 0x7FFFu;
    if (mag == 0) return s ? -0.0 : 0.0;
    const int lead = (mag >> 14) & 1;
    int run = 0, pos = 14;
    while (pos >= 0 && (int)((mag >> pos) & 1u) == lead) { ++run; --pos; }
    const int k = lead ? run - 1 : -run;
    const int avail = pos > 0 ? pos : 0;          /* bits below the terminating bit */
    const int ebits = std::min(es, avail);
    int e = ebits ? (int)((mag >> (avail - ebits)) & ((1u << ebits) - 1u)) : 0;
    e <<= (es - ebits);                           /* missing low exponent bits are zero */
    const int nf = avail - ebits;
    const uint32_t frac = mag & ((1u << nf) - 1u);
    const double v = std::ldexp(1.0 + std::ldexp((double)frac, -nf), k * (1 << es) + e);
    return s ? -v : v;
}

/* Value of the asymmetric P16_2C posit: v leading zeros, a terminating one,
 * two exponent bits, 12-v fraction bits; value 2^(-4v + e - 3) (1 + fraction). */
double p162c_value(uint16_t c) {
    const int s = c >> 15;
    const uint32_t mag = c & 0x7FFFu;
    if (mag == 0) return s ? -0.0 : 0.0;
    int v = 0;
    while (!((mag >> (14 - v)) & 1u)) ++v;
    const int avail = 14 - v;
    int e = 0, nf = 0;
    if (avail >= 2) { e = (int)((mag >> (avail - 2)) & 3u); nf = avail - 2; }
    const uint32_t frac = mag & ((1u << nf) - 1u);
    const double val = std::ldexp(1.0 + std::ldexp((double)frac, -nf), -4 * v + e - 3);
    return s ? -val : val;
}

/* Magnitude tables of the posit formats (codes 0..0x7FFF, non-decreasing). */
struct Table { std::vector<double> v; };
const Table& table(int which) {
    static Table t[3];
    static std::once_flag once;
    std::call_once(once, [] {
        for (int w = 0; w < 3; ++w) {
            t[w].v.resize(0x8000);
            for (uint32_t c = 0; c < 0x8000u; ++c)
                t[w].v[c] = (w == 2) ? p162c_value((uint16_t)c) : posit_sm_value((uint16_t)c, w);
        }
    });
    return t[which];
}

/* lowest code whose magnitude equals the representable value r */
uint16_t code_of(int which, double r) {
    const std::vector<double>& v = table(which).v;
    return (uint16_t)(std::lower_bound(v.begin(), v.end(), r) - v.begin());
}

/* P16_0: values 2^-14 .. 2^14.  Rounding: nearest value (binade-uniform
 * spacing), ties away from zero; zero below 2^-15 (half of the smallest
 * value); saturation from 2^14 upward; NaN saturates with its sign. */
uint16_t p160_from_float(float y) {
    const uint16_t s = (uint16_t)((fbits(y) >> 16) & 0x8000u);
    const double a = std::fabs((double)y);
    if (std::isnan(y) || a >= 0x1p14) return (uint16_t)(s | 0x7FFFu);
    if (a < 0x1p-15) return s;
    if (a < 0x1p-14) return (uint16_t)(s | 1u);
    const int E = ilog2(a);                             /* -14 .. 13, regime k = E */
    const int nf = E >= 0 ? 13 - E : 14 + E;            /* fraction bits in this binade */
    return (uint16_t)(s | code_of(0, round_half_up_binade(a, E, nf)));
}

/* P16_1: values 2^-28 .. 2^28.  Between 2^-26 and 2^26: nearest value, ties
 * away from zero.  Where the exponent bit no longer fits below the regime the
 * rounding follows the bit string (midpoints at odd powers of two):
 *   [2^-30, 2^-27) -> 2^-28,  [2^-27, 2^-26) -> 2^-26,
 *   [2^26, 2^27)   -> 2^26,   [2^27, inf]    -> 2^28;   below 2^-30: zero. */
uint16_t p161_from_float(float y) {
    const uint16_t s = (uint16_t)((fbits(y) >> 16) & 0x8000u);
    const double a = std::fabs((double)y);
    if (std::isnan(y) || a >= 0x1p27) return (uint16_t)(s | 0x7FFFu);
    if (a >= 0x1p26) return (uint16_t)(s | 0x7FFEu);
    if (a < 0x1p-30) return s;
    if (a < 0x1p-27) return (uint16_t)(s | 1u);
    if (a < 0x1p-26) return (uint16_t)(s | 2u);
    const int E = ilog2(a);                             /* -26 .. 25 */
    const int k = (E >= 0) ? E / 2 : -((-E + 1) / 2);   /* floor(E/2) */
    const int nf = k >= 0 ? 12 - k : 13 + k;
    return (uint16_t)(s | code_of(1, round_half_up_binade(a, E, nf)));
}

/* P16_2C: values 2^-59 .. 1.999756.  Between 2^-51 and 2: nearest value,
 * ties away from zero.  Rules at the ends:
 *   [2^-53, 2^-51) -> code 4 (2^-51)
 *   [2^-55, 2^-53) -> code 3, [2^-58, 2^-55) -> code 2 (both decode to 2^-55)
 *   below 2^-58 -> zero;  2 and above, NaN -> saturate (0x7FFF);
 *   [2 - 2^-13, 2): the rounding carry leaves the 15-bit field -> zero. */
uint16_t p162c_from_float(float x) {
    const uint16_t s = (uint16_t)((fbits(x) >> 16) & 0x8000u);
    const double a = std::fabs((double)x);
    if (std::isnan(x) || a >= 2.0) return (uint16_t)(s | 0x7FFFu);
    if (a < 0x1p-58) return s;
    if (a < 0x1p-55) return (uint16_t)(s | 2u);
    if (a < 0x1p-53) return (uint16_t)(s | 3u);
    if (a < 0x1p-51) return (uint16_t)(s | 4u);
    const int E = ilog2(a);                             /* -51 .. 0 */
    const int v = (-E) / 4;                             /* regime zeros */
    const double r = round_half_up_binade(a, E, 12 - v);
    if (r >= 2.0) return s;
    return (uint16_t)(s | code_of(2, r));
}

float decode_value(int fmt, uint16_t c) {
    switch (fmt) {
    case ORC_FP16:   return (float)fp16_value(c);
    case ORC_FP16S:  return (float)fp16_value(c) * 3.0517578E-5f;   /* 2^-15 in FP32 */
    case ORC_FP16C:  return (float)fp16c_value(c);
    case ORC_P16_0S: return (float)posit_sm_value(c, 0) * 0.0078125f; /* 2^-7 */
    case ORC_P16_1S: return (float)posit_sm_value(c, 1) * 0.0078125f;
    case ORC_P16_2C: return (float)p162c_value(c);
    case ORC_P16_0:  return (float)posit_sm_value(c, 0);
    case ORC_P16_1:  return (float)posit_sm_value(c, 1);
    default:         return NAN;
    }
}

/* posit formats: a NaN saturates with the sign of the input (the scaling
 * product of the S variants is not consulted, since hardware may return a
 * NaN of either sign for NaN * 128) */
uint16_t nan_code(float x) { return (uint16_t)(((fbits(x) >> 16) & 0x8000u) | 0x7FFFu); }

uint16_t encode_value(int fmt, float x) {
    switch (fmt) {
    case ORC_FP16:   return fp16_from_float(x);
    case ORC_FP16S:  return fp16_from_float(x * 32768.0f);        /* FP32 product */
    case ORC_FP16C:  return fp16c_from_float(x);
    case ORC_P16_0S: return std::isnan(x) ? nan_code(x) : p160_from_float(x * 128.0f);
    case ORC_P16_1S: return std::isnan(x) ? nan_code(x) : p161_from_float(x * 128.0f);
    case ORC_P16_2C: return p162c_from_float(x);
    case ORC_P16_0:  return p160_from_float(x);
    case ORC_P16_1:  return p161_from_float(x);
    default:         return 0;
    }
}

}  // namespace

extern "C" {

uint16_t orc_encode(int fmt, float x) { return encode_value(fmt, x); }
float orc_decode(int fmt, uint16_t c) { return decode_value(fmt, c); }

void orc_encode_array(int fmt, const float* x, uint16_t* out, int64_t n) {
    table(0);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) out[i] = encode_value(fmt, x[i]);
}

void orc_decode_array(int fmt, const uint16_t* c, float* out, int64_t n) {
    for (int64_t i = 0; i < n; ++i) out[i] = decode_value(fmt, c[i]);
}

void orc_encode_bits_range(int fmt, uint32_t first, int64_t n, uint16_t* out) {
    table(0);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        const uint32_t b = first + (uint32_t)i;
        float x;
        std::memcpy(&x, &b, 4);
        out[i] = encode_value(fmt, x);
    }
}

}  // extern "C"
