// Device building blocks of the stream-collide step (arXiv 2112.08926):
// velocity sets, storage codecs of Sec. 3, and the collision of Sec. 2.2 in
// the operation order the paper prescribes.  Compiled with --fmad=false, so
// every fused multiply-add below is an explicit fma() and nothing else fuses.
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

#include <type_traits>

namespace lbm {

// Compile-time loop: calls f(std::integral_constant<int, I>) for I = B..E-1,
// so direction indices, velocities and weights are constant expressions.
template <int B, int E, class F>
__host__ __device__ __forceinline__ void static_for(F&& f) {
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        static_for<B + 1, E>(f);
    }
}

enum : uint32_t {
    F_WALL = 0x01u, F_MOVING = 0x02u, F_EQ = 0x04u, F_OUTFLOW = 0x08u, F_FREESLIP = 0x10u
};

// ---------------------------------------------------------------- velocity sets
// Direction convention: 0 rest, (2k-1, 2k) opposite pairs.  D3Q19 follows the
// paper's D3Q19 core; D3Q27 appends the corners.
struct D2Q9 {
    static constexpr int Q = 9, D = 2, ID = 0;
    __host__ __device__ static constexpr int c(int i, int a) {
        constexpr int t[9][3] = {{0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0},
                                 {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}};
        return t[i][a];
    }
    __host__ __device__ static constexpr double w(int i) {
        return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
};

struct D3Q27 {
    static constexpr int Q = 27, D = 3, ID = 2;
    __host__ __device__ static constexpr int c(int i, int a) {
        constexpr int t[27][3] = {
            {0, 0, 0},
            {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
            {1, 1, 0}, {-1, -1, 0}, {1, 0, 1}, {-1, 0, -1}, {0, 1, 1}, {0, -1, -1},
            {1, -1, 0}, {-1, 1, 0}, {1, 0, -1}, {-1, 0, 1}, {0, 1, -1}, {0, -1, 1},
            {1, 1, 1}, {-1, -1, -1}, {1, 1, -1}, {-1, -1, 1},
            {1, -1, 1}, {-1, 1, -1}, {-1, 1, 1}, {1, -1, -1}};
        return t[i][a];
    }
    __host__ __device__ static constexpr double w(int i) {
        return i == 0 ? 8.0 / 27.0 : (i < 7 ? 2.0 / 27.0 : (i < 19 ? 1.0 / 54.0 : 1.0 / 216.0));
    }
};

struct D3Q19 {
    static constexpr int Q = 19, D = 3, ID = 1;
    __host__ __device__ static constexpr int c(int i, int a) { return D3Q27::c(i, a); }
    __host__ __device__ static constexpr double w(int i) {
        return i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0);
    }
};

__host__ __device__ constexpr int opposite(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }

// direction whose velocity is c_i with component `axis` reversed
template <class V>
__host__ __device__ constexpr int mirror(int i, int axis) {
    int r = i;
    for (int j = 0; j < V::Q; ++j) {
        bool same = true;
        for (int a = 0; a < 3; ++a) {
            const int want = (a == axis) ? -V::c(i, a) : V::c(i, a);
            if (V::c(j, a) != want) same = false;
        }
        if (same) r = j;
    }
    return r;
}

// ---------------------------------------------------------------- storage codecs
// Every storage type provides load (code -> arithmetic value) and store
// (arithmetic value -> code).  The 16-bit codecs are bit-level designs for
// sm_103a written from the format definitions of Sec. 3; they produce the same
// codes as the paper's conversion routines but with fewer instructions.

__device__ __forceinline__ uint32_t u32(float x) { return __float_as_uint(x); }

// FP16C (1|4|11, bias 15, Sec. 3.1.2): place the 15 magnitude bits under an
// FP32 exponent field and multiply by 2^112; exponent 0 lands in the FP32
// subnormal range and scales to the FP16C subnormals exactly (needs no FTZ).
__device__ __forceinline__ float fp16c_decode(uint32_t c) {
    const uint32_t b = ((c & 0x8000u) << 16) | ((c & 0x7FFFu) << 12);
    return __uint_as_float(b) * 0x1p112f;
}

// FP32 -> FP16C: round to nearest, halfway cases away from zero, subnormals
// kept, saturation at the largest magnitude.  |x| * 2^-112 (rounded toward
// zero) puts the FP16C exponent range onto FP32 exponents 1..15 and the FP16C
// subnormals onto FP32 subnormals, truncated to whole units of 2^-149 = 2^-37
// in FP16C terms; adding half a unit of bit 12 and dropping 12 bits then
// rounds half up in both ranges at once (the truncation cannot move a value
// across a halfway point, which lies on the 2^-149 grid).  NaN patterns whose
// rounding increment would carry into the sign give a zero of the opposite
// sign.
__device__ __forceinline__ uint32_t fp16c_encode(float x) {
    const uint32_t b = u32(x);
    const uint32_t a = b & 0x7FFFFFFFu;
    const float y = __fmul_rz(__uint_as_float(a), 0x1p-112f);
    const uint32_t code = min((u32(y) + 0x800u) >> 12, 0x7FFFu);
    const uint32_t s = (b >> 16) & 0x8000u;
    return a >= 0x7FFFF800u ? (s ^ 0x8000u) : (s | code);
}

// Posits (Sec. 3.2): a 15-bit magnitude under the sign bit.  P16_0 / P16_1:
// a regime run (r+1 ones and a zero for r >= 0, -r zeros and a one for r < 0),
// ES exponent bits, the fraction; value 2^(r 2^ES + e) (1 + fraction).
// P16_2C (asymmetric, lower flank only): v zeros and a one, two exponent
// bits, the fraction; value 2^(-4v + e - 3) (1 + fraction).  All conversions
// below are branch-free.

// Decode: the run of bits equal to bit 14 becomes leading zeros (xor with the
// sign-extended bit 14) and is counted in one instruction; the bits after the
// terminator, moved to the top of a word, hold the exponent bits and the
// fraction, and one addition puts them under the regime's exponent.  Exponent
// bits cut off by a long regime read as zero.  bias_shift folds the 2^-7
// decode scale of the S variants into the exponent (exact).  A zero magnitude
// decodes to +-0.
template <int ES>
__device__ __forceinline__ float posit_decode(uint32_t c, int bias_shift) {
    const uint32_t x = c << 17;                                  // magnitude in bits 31..17
    const uint32_t m = (uint32_t)((int32_t)x >> 31);             // all ones for a run of ones
    const int n = __clz(x ^ m);                                  // run length (32: zero magnitude)
    const int k = (n - 1) ^ (int)~m;                             // regime: n - 1 (ones), -n (zeros)
    const uint32_t r = __funnelshift_lc(0u, x, (uint32_t)n + 1u);   // the bits after the terminator
    const uint32_t bits = ((uint32_t)k << (23 + ES)) + ((uint32_t)(127 + bias_shift) << 23) + (r >> (9 - ES));
    const uint32_t sign = (c & 0x8000u) << 16;
    return __uint_as_float(x ? (bits | sign) : sign);
}

// P16_2C: with 13 leading zeros only one exponent bit fits, and it reads as
// zero (the exponent bits cut off by the regime); 14 zeros leave none.
__device__ __forceinline__ float p162c_decode(uint32_t c) {
    const uint32_t x = c << 17;
    const uint32_t v = (uint32_t)__clz(x);                       // leading zeros (32: zero magnitude)
    uint32_t r = __funnelshift_lc(0u, x, v + 1u);                // exponent bits and fraction at the top
    r = v < 13u ? r : 0u;
    const uint32_t bits = (124u << 23) - (v << 25) + (r >> 7);   // exponent field 124 - 4v + e
    const uint32_t sign = (c & 0x8000u) << 16;
    return __uint_as_float(x ? (bits | sign) : sign);
}

// Encode P16_0 / P16_1: the bit string of |y| -- regime, exponent bit, the 23
// FP32 mantissa bits -- is laid out in one word below the regime's first bit
// (the run of ones of a regime r >= 0 comes from sign extension), shifted so
// that 16 bits remain, and the last of them (the first bit cut off) is
// added: nearest value with ties away from zero where fraction bits fit, and
// rounding of the bit string where the regime leaves no room for the
// exponent bit.  Magnitudes from the largest code on, Inf and NaN saturate;
// zeros, FP32 subnormals and values below half the smallest code give 0.
// The sign of y is copied.
template <int ES>
__device__ __forceinline__ uint32_t posit_encode(float y) {
    const uint32_t b = u32(y);
    const int E = (int)((b >> 23) & 0xFFu) - 127;
    const int k = min(E >> ES, 14);                              // regime floor(E / 2^ES), saturating
    const uint32_t neg = (uint32_t)(k >> 31);                    // all ones for r < 0
    // exponent bit and mantissa; for ES = 1 the exponent bit is the FP32
    // exponent's low bit inverted (E = field - 127, 127 odd)
    const uint32_t t = ES == 1 ? ((b ^ 0x00800000u) & 0x00FFFFFFu) : (b & 0x007FFFFFu);
    // terminator at bit 23 + ES: a one under zeros (r < 0), a zero under ones
    const uint32_t X = t + (neg & (3u << (23 + ES))) + (0xFFFFFFFFu << (24 + ES));
    const uint32_t sh = (uint32_t)(k ^ (int)neg) + (uint32_t)(9 + ES);   // leaves field + rounding bit
    const uint32_t w = __funnelshift_rc(X, ~neg, sh);            // X >> sh, sign-extended, clamped
    return ((b >> 16) & 0x8000u) | (((w + 1u) >> 1) & 0x7FFFu);
}

// Encode P16_2C: the same with v = floor(-E / 4) zeros and the exponent field
// 3 - (-E mod 4); a carry out of the 15 bits (just below 2) leaves 0.  End
// rules: from 2 on (and NaN) saturation; below 2^-51 the printed conversion's
// own rounding of the lowest numbers: [2^-53, 2^-51) -> 4, [2^-55, 2^-53) -> 3,
// [2^-58, 2^-55) -> 2, smaller -> 0.
__device__ __forceinline__ uint32_t p162c_encode(float x) {
    const uint32_t b = u32(x);
    const int E = (int)((b >> 23) & 0xFFu) - 127;
    const uint32_t ae = (uint32_t)max(-E, 0);
    const uint32_t X = 0x02000000u | ((~ae & 3u) << 23) | (b & 0x007FFFFFu);
    const uint32_t w = X >> min((ae >> 2) + 10u, 31u);
    uint32_t mag = ((w + 1u) >> 1) & 0x7FFFu;
    mag = E >= 1 ? 0x7FFFu : mag;
    mag = E < -51 ? (E >= -53 ? 4u : (E >= -55 ? 3u : (E >= -58 ? 2u : 0u))) : mag;
    return ((b >> 16) & 0x8000u) | mag;
}

// Table-driven posit encoder (used where a block holds the table in shared
// memory).  Within one FP32 binade of |y| the code is linear in |y| (where
// fraction bits fit) or constant (where the regime cuts exponent bits off,
// and at the ends of the range), so one fused multiply-add rounded toward
// zero gives it: with s = 2^(nf - E) (nf fraction bits) and o = 2^22 + c0 -
// 2^nf + 1/2 (c0 the code of 2^E), fma_rz(|y|, s, o) = 2^22 + c0 +
// floor(f 2^nf + 1/2) + {0, 1/2} in [2^22, 2^23), whose mantissa holds the
// code above one bit of the half.  The entries are indexed by the sign and the
// exponent field of y (s is negated for negative y).  Inf and NaN give NaN,
// whose pattern 0x7FFFFFFF holds the largest code.
struct EncEntry {
    float s, o;
};
struct EncTable {
    EncEntry e[512];
};

// constexpr 2^n as float (|n| < 128)
__host__ __device__ constexpr float pow2f(int n) {
    double v = 1.0;
    for (int i = 0; i < (n < 0 ? -n : n); ++i) v = n < 0 ? v * 0.5 : v * 2.0;
    return (float)v;
}

// FMT: 5..9 (the table works on the value as stored, times 2^SL for the S
// variants, like enc_g)
template <int FMT>
__host__ __device__ constexpr EncTable make_enc_table() {
    constexpr bool asym = FMT == 7;
    constexpr int ES = (FMT == 5 || FMT == 8) ? 0 : (FMT == 7 ? 2 : 1);
    EncTable t{};
    for (int e9 = 0; e9 < 512; ++e9) {
        const int e8 = e9 & 255;
        const float sgn = e9 >= 256 ? -1.0f : 1.0f;
        const int E = e8 - 127;
        long long cst = -1;   // constant code, or -1 for a linear binade
        int nf = 0;
        long long c0 = 0;
        if (e8 == 0) {
            cst = 0;
        } else if (e8 == 255) {
            cst = 0x7FFF;
        } else if (asym) {
            if (E >= 1) cst = 0x7FFF;
            else if (E < -51) cst = E >= -53 ? 4 : (E >= -55 ? 3 : (E >= -58 ? 2 : 0));
            else {
                const int v = (-E) >> 2, ee = 3 - ((-E) & 3);
                nf = 12 - v;
                c0 = (1ll << (14 - v)) | ((long long)ee << nf);
            }
        } else if (E >= (14 << ES)) {
            cst = 0x7FFF;
        } else {
            const int k = E >= 0 ? (E >> ES) : -((-E + (1 << ES) - 1) >> ES);   // floor(E / 2^ES)
            const int ee = E - k * (1 << ES);
            const int rl = k >= 0 ? k + 2 : 1 - k;                               // regime bits with terminator
            const long long reg = k >= 0 ? (((1ll << (k + 1)) - 1) << 1) : 1ll;
            nf = 15 - rl - ES;
            if (nf >= 0) {
                c0 = (reg << (15 - rl)) | ((long long)ee << nf);
            } else {
                const long long str = (reg << ES) | ee;                         // rl + ES > 15 bits
                const int L = rl + ES;
                cst = L > 40 ? 0 : (str >> (L - 15)) + ((str >> (L - 16)) & 1);
            }
        }
        if (cst >= 0) {
            t.e[e9].s = 0.0f;
            t.e[e9].o = pow2f(22) + (float)cst + 0.5f;
        } else {
            t.e[e9].s = sgn * pow2f(nf - E);
            t.e[e9].o = pow2f(22) + (float)(c0 - (1ll << nf)) + 0.5f;
        }
    }
    return t;
}

// the encoding table of each posit format, in device memory (copied into
// shared memory by the kernels that use it)
template <int FMT> __device__ const EncTable kEncTable = make_enc_table<FMT>();

// the code of g (scaled as stored) from a table entry
__device__ __forceinline__ uint32_t enc_table(const EncEntry* tab, float g) {
    const uint32_t b = u32(g);
    const EncEntry t = tab[b >> 23];
    const uint32_t v = u32(__fmaf_rz(g, t.s, t.o));
    return ((v >> 1) & 0x7FFFu) | ((b >> 16) & 0x8000u);
}
// two codes as one pair (lo in bits 0..15, hi in bits 16..31)
__device__ __forceinline__ uint32_t enc_table_pair(const EncEntry* tab, float lo, float hi) {
    const uint32_t bl = u32(lo), bh = u32(hi);
    const EncEntry tl = tab[bl >> 23], th = tab[bh >> 23];
    const uint32_t vl = u32(__fmaf_rz(lo, tl.s, tl.o)), vh = u32(__fmaf_rz(hi, th.s, th.o));
    const uint32_t c = __byte_perm(vl >> 1, vh << 15, 0x7610);   // codes at bits 0..14 and 16..30
    const uint32_t sg = __byte_perm(bl, bh, 0x7030);             // sign bits at 15 and 31
    return (c & 0x7FFF7FFFu) | (sg & 0x80008000u);
}

// Codec16<FMT>: dec/enc convert between a code and the population value;
// dec_g/enc_g work on the value times 2^SL, the scale the S formats apply
// before encoding (Sec. 3.1.3, 3.2.2), so a kernel that keeps its populations
// scaled skips both multiplications.  Scaling by a power of two commutes with
// rounding, so either route gives the same codes.
template <int FMT> struct Codec16;
template <> struct Codec16<2> {   // FP16: IEEE binary16, round to nearest even (hardware)
    static constexpr int SL = 0;
    __device__ static float dec_g(uint32_t c) { return __half2float(__ushort_as_half((unsigned short)c)); }
    __device__ static uint32_t enc_g(float g) { return __half_as_ushort(__float2half_rn(g)); }
    __device__ static float dec(uint32_t c) { return dec_g(c); }
    __device__ static uint32_t enc(float x) { return enc_g(x); }
};
template <> struct Codec16<3> {   // FP16S: binary16 of x * 2^15 (Sec. 3.1.3)
    static constexpr int SL = 15;
    __device__ static float dec_g(uint32_t c) { return __half2float(__ushort_as_half((unsigned short)c)); }
    __device__ static uint32_t enc_g(float g) { return __half_as_ushort(__float2half_rn(g)); }
    __device__ static float dec(uint32_t c) { return dec_g(c) * 3.0517578125e-5f; }
    __device__ static uint32_t enc(float x) { return enc_g(x * 32768.0f); }
};
template <> struct Codec16<4> {   // FP16C (Sec. 3.1.4)
    static constexpr int SL = 0;
    __device__ static float dec_g(uint32_t c) { return fp16c_decode(c); }
    __device__ static uint32_t enc_g(float g) { return fp16c_encode(g); }
    __device__ static float dec(uint32_t c) { return dec_g(c); }
    __device__ static uint32_t enc(float x) { return enc_g(x); }
};
// The S posits encode |x| * 2^7 with the sign of x itself, so a NaN
// saturates with its own sign whatever sign the hardware gives NaN * 128.
template <> struct Codec16<5> {   // P16_0S: posit es=0 of x * 2^7
    static constexpr int SL = 7;
    __device__ static float dec_g(uint32_t c) { return posit_decode<0>(c, 0); }
    __device__ static uint32_t enc_g(float g) { return posit_encode<0>(g); }
    __device__ static float dec(uint32_t c) { return posit_decode<0>(c, -7); }
    __device__ static uint32_t enc(float x) {
        return posit_encode<0>(fabsf(x) * 128.0f) | ((u32(x) >> 16) & 0x8000u);
    }
};
template <> struct Codec16<6> {   // P16_1S: posit es=1 of x * 2^7
    static constexpr int SL = 7;
    __device__ static float dec_g(uint32_t c) { return posit_decode<1>(c, 0); }
    __device__ static uint32_t enc_g(float g) { return posit_encode<1>(g); }
    __device__ static float dec(uint32_t c) { return posit_decode<1>(c, -7); }
    __device__ static uint32_t enc(float x) {
        return posit_encode<1>(fabsf(x) * 128.0f) | ((u32(x) >> 16) & 0x8000u);
    }
};
template <> struct Codec16<7> {   // P16_2C
    static constexpr int SL = 0;
    __device__ static float dec_g(uint32_t c) { return p162c_decode(c); }
    __device__ static uint32_t enc_g(float g) { return p162c_encode(g); }
    __device__ static float dec(uint32_t c) { return dec_g(c); }
    __device__ static uint32_t enc(float x) { return enc_g(x); }
};
template <> struct Codec16<8> {   // P16_0, unscaled
    static constexpr int SL = 0;
    __device__ static float dec_g(uint32_t c) { return posit_decode<0>(c, 0); }
    __device__ static uint32_t enc_g(float g) { return posit_encode<0>(g); }
    __device__ static float dec(uint32_t c) { return dec_g(c); }
    __device__ static uint32_t enc(float x) { return enc_g(x); }
};
template <> struct Codec16<9> {   // P16_1, unscaled
    static constexpr int SL = 0;
    __device__ static float dec_g(uint32_t c) { return posit_decode<1>(c, 0); }
    __device__ static uint32_t enc_g(float g) { return posit_encode<1>(g); }
    __device__ static float dec(uint32_t c) { return dec_g(c); }
    __device__ static uint32_t enc(float x) { return enc_g(x); }
};

// Storage traits: FMT is the lbm.h storage id.  load/store handle population
// values; load_g/store_g handle values scaled by 2^SL (see Codec16).
template <int FMT> struct Storage {
    using T = uint16_t;
    static constexpr int bytes = 2;
    static constexpr int SL = Codec16<FMT>::SL;
    template <class R, class IX> __device__ static R load_g(const T* p, IX i) { return (R)Codec16<FMT>::dec_g(p[i]); }
    template <class R, class IX> __device__ static void store_g(T* p, IX i, R g) {
        p[i] = (uint16_t)Codec16<FMT>::enc_g((float)g);
    }
    template <class R, class IX> __device__ static R load(const T* p, IX i) { return (R)Codec16<FMT>::dec(p[i]); }
    template <class R, class IX> __device__ static void store(T* p, IX i, R v) {
        p[i] = (uint16_t)Codec16<FMT>::enc((float)v);
    }
};
template <> struct Storage<0> {   // FP64
    using T = double;
    static constexpr int bytes = 8;
    static constexpr int SL = 0;
    template <class R, class IX> __device__ static R load(const T* p, IX i) { return (R)p[i]; }
    template <class R, class IX> __device__ static void store(T* p, IX i, R v) { p[i] = (double)v; }
    template <class R, class IX> __device__ static R load_g(const T* p, IX i) { return (R)p[i]; }
    template <class R, class IX> __device__ static void store_g(T* p, IX i, R v) { p[i] = (double)v; }
};
// FP32 <-> FP64 on the integer pipe.  On GB300 the FP64 pipe bounds the
// FP64-arithmetic tiers, and the hardware conversions run there too, so the
// FP64/FP32 tier converts in integer arithmetic (IEEE 754 binary32 and
// binary64 encodings; round to nearest even).  Zeros are handled here; the
// rare cases outside the normal range of the result go to the hardware.
__device__ __forceinline__ double f32_to_f64(float x) {
    const uint32_t b = __float_as_uint(x);
    const uint32_t mag = b & 0x7FFFFFFFu;
    if (mag == 0u) return __hiloint2double((int)(b & 0x80000000u), 0);
    if ((mag >> 23) - 1u >= 254u) return (double)x;   // subnormal, Inf, NaN
    // exponent + (1023 - 127) in the high word, mantissa split across both words
    const uint32_t hi = (b & 0x80000000u) | ((mag >> 3) + 0x38000000u);
    return __hiloint2double((int)hi, (int)(b << 29));
}
__device__ __forceinline__ float f64_to_f32(double v) {
    const uint32_t hi = (uint32_t)__double2hiint(v), lo = (uint32_t)__double2loint(v);
    const uint32_t e = (hi >> 20) & 0x7FFu;
    if (((hi & 0x7FFFFFFFu) | lo) == 0u) return __uint_as_float(hi & 0x80000000u);
    if (e - 897u >= 254u) return (float)v;            // result subnormal, zero, huge, Inf or NaN
    // 23-bit mantissa and exponent - (1023 - 127): the upper word of (hi:lo) << 3
    // minus 896 << 23 (mod 2^32; the exponent's bits above bit 31 cancel)
    const uint32_t m = __funnelshift_l(lo, hi, 3) - 0xC0000000u;
    const uint32_t rem = lo & 0x1FFFFFFFu;          // the 29 dropped bits
    const uint32_t up = (rem > 0x10000000u || (rem == 0x10000000u && (m & 1u))) ? 1u : 0u;
    return __uint_as_float((hi & 0x80000000u) | (m + up));
}
template <class R> __device__ __forceinline__ R from_f32(float x) {
    if constexpr (sizeof(R) == 8) return f32_to_f64(x); else return x;
}
template <class R> __device__ __forceinline__ float to_f32(R v) {
    if constexpr (sizeof(R) == 8) return f64_to_f32(v); else return v;
}

template <> struct Storage<1> {   // FP32
    using T = float;
    static constexpr int bytes = 4;
    static constexpr int SL = 0;
    template <class R, class IX> __device__ static R load(const T* p, IX i) { return from_f32<R>(p[i]); }
    template <class R, class IX> __device__ static void store(T* p, IX i, R v) { p[i] = to_f32(v); }
    template <class R, class IX> __device__ static R load_g(const T* p, IX i) { return from_f32<R>(p[i]); }
    template <class R, class IX> __device__ static void store_g(T* p, IX i, R v) { p[i] = to_f32(v); }
};

// ---------------------------------------------------------------- collision
__device__ __forceinline__ float fmaR(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmaR(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float minR(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double minR(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ float maxR(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double maxR(double a, double b) { return fmax(a, b); }

// Relaxation constants in arithmetic precision (computed on the host).
// sh is the DDF shift (Sec. 2.2): 1 when populations are stored as f - w,
// 0 for the unshifted ablation (appendix, "without DDF-shifting"), where the
// same formulas with rho = sum f and D = w rho give the plain equilibrium.
template <class R> struct Relax {
    R om, c1, omp, omm, cSp, cSm, cs;
    R omph, ommh, cSph, cSmh;   // TRT: omega+/2, omega-/2, (1 - omega+/2)/2, (1 - omega-/2)/2 (exact halves)
    R F[3];
    R sh;
    int force;
    int xsafe;                // every F_a is 0 or 2^-76 <= |F_a| <= 2^90 (see numerators_ok)
    R mrt_r[19], mrt_p[19];   // MRT: s_k / |M_k|^2 and (1 - s_k / 2) / |M_k|^2 (D3Q19)
};

// D3Q19 multiple-relaxation-time basis (d'Humieres et al. 2002): moment k of
// direction i as a velocity polynomial -- rho, e, epsilon, j_x, q_x, j_y,
// q_y, j_z, q_z, 3 p_xx, 3 pi_xx, p_ww, pi_ww, p_xy, p_yz, p_xz, m_x, m_y,
// m_z.  Every entry is an integer.
template <class V>
__host__ __device__ constexpr int mrt_m(int k, int i) {
    const int x = V::c(i, 0), y = V::c(i, 1), z = V::c(i, 2), c2 = x * x + y * y + z * z;
    switch (k) {
    case 0: return 1;
    case 1: return 19 * c2 - 30;
    case 2: return (21 * c2 * c2 - 53 * c2 + 24) / 2;
    case 3: return x;
    case 4: return (5 * c2 - 9) * x;
    case 5: return y;
    case 6: return (5 * c2 - 9) * y;
    case 7: return z;
    case 8: return (5 * c2 - 9) * z;
    case 9: return 3 * x * x - c2;
    case 10: return (3 * c2 - 5) * (3 * x * x - c2);
    case 11: return y * y - z * z;
    case 12: return (3 * c2 - 5) * (y * y - z * z);
    case 13: return x * y;
    case 14: return y * z;
    case 15: return x * z;
    case 16: return x * (y * y - z * z);
    case 17: return y * (z * z - x * x);
    default: return z * (x * x - y * y);
    }
}

// sum over axes of c_ia * v_a in axis order: the first non-zero term is +-v_a,
// each later one is added or subtracted (no multiplications)
template <class V, int I, class R>
__device__ __forceinline__ R csum(const R* v) {
    constexpr int c0 = V::c(I, 0), c1 = V::c(I, 1), c2 = V::c(I, 2);
    R s = R(0);
    if constexpr (c0 != 0) s = c0 > 0 ? v[0] : -v[0];
    if constexpr (c1 != 0) {
        if constexpr (c0 == 0) s = c1 > 0 ? v[1] : -v[1];
        else s = c1 > 0 ? s + v[1] : s - v[1];
    }
    if constexpr (c2 != 0) {
        if constexpr (c0 == 0 && c1 == 0) s = c2 > 0 ? v[2] : -v[2];
        else s = c2 > 0 ? s + v[2] : s - v[2];
    }
    return s;
}

// alternating-sign momentum sum along axis A over the pairs p..Q-1 (p odd),
// continuing the running sum s (first: no term yet)
template <class V, int A, int P, bool FIRST, class R>
__device__ __forceinline__ R jsum(const R* f, R s) {
    if constexpr (P >= V::Q) {
        return s;
    } else {
        constexpr int ca = V::c(P, A);
        if constexpr (ca == 0) {
            return jsum<V, A, P + 2, FIRST, R>(f, s);
        } else {
            constexpr int pos = ca > 0 ? P : P + 1;
            constexpr int neg = ca > 0 ? P + 1 : P;
            if constexpr (FIRST) return jsum<V, A, P + 2, false, R>(f, f[pos] - f[neg]);
            else return jsum<V, A, P + 2, false, R>(f, (s + f[pos]) - f[neg]);
        }
    }
}

// 2^SL and 2^-SL as exact constants
template <int SL> struct Pow2 {
    static constexpr double up = (double)(1ull << SL);
    static constexpr double down = 1.0 / (double)(1ull << SL);
};

// Populations g = 2^SL f (SL = 0: unscaled).  Density in index order with 1
// added last (Sec. 2.2): rho = (sum f) + 1, the exact sum of the scaled
// values times 2^-SL being fused into that last addition; the momentum j is
// returned scaled (alternating-sign sums over opposite pairs, Sec. 2.2).
// sh = 0 (unshifted populations) adds nothing.
template <class V, class R, int SL>
__device__ __forceinline__ void moments(const R* g, R& rho, R* j, R sh) {
    R s = g[0];
    static_for<1, V::Q>([&](auto I) { s = s + g[I.value]; });
    if constexpr (SL == 0) rho = s + sh;
    else rho = fmaR(s, R(Pow2<SL>::down), sh);
    j[0] = jsum<V, 0, 1, true, R>(g, R(0));
    j[1] = jsum<V, 1, 1, true, R>(g, R(0));
    j[2] = jsum<V, 2, 1, true, R>(g, R(0));
}

// Velocity u_a = x_a / rho with x_a = j_a + F_a/2 (Sec. 2.2: each momentum
// component divided by rho, u_x = (f1 - f2 + ...)/rho; Guo half-force), before
// clamping, as the IEEE quotient of each component.  It is computed from one
// IEEE reciprocal y = 1/rho (rounded to nearest) by two FMA corrections:
//   q0 = x y;  q1 = q0 + (x - rho q0) y;  u = q1 + (x - rho q1) y.
// q0 can lie up to 1.5 ulp off x/rho; after the first correction q1 is within
// one ulp (faithful), so x - rho q1 is exact, and by Markstein's theorem
// (P. Markstein, IBM J. Res. Dev. 34 (1990) 111: a faithful quotient
// corrected with the correctly rounded reciprocal) u is the correctly rounded
// quotient -- provided nothing overflows and no residual falls below the
// normal range.  A residual of a faithful quotient is a multiple of
// ulp(q) ulp(rho) >= 2^(e_x - 47), so |x| in [2^-100, 2^100] with rho in
// [2^-20, 2^20] keeps every intermediate normal and exact (FP64: 2^-800,
// 2^800 and 2^-200, 2^200).  A zero x gives a zero of the right sign once the
// sign of x is copied back.  Outside those ranges the IEEE division itself is
// taken.  (Three IEEE divisions give the same bits; on lattices at rest they
// ran much slower.)
template <class R> struct DivRange;
template <> struct DivRange<float> {
    static constexpr float xlo = 0x1p-100f, xhi = 0x1p100f, rlo = 0x1p-20f, rhi = 0x1p20f;
};
template <> struct DivRange<double> {
    static constexpr double xlo = 0x1p-800, xhi = 0x1p800, rlo = 0x1p-200, rhi = 0x1p200;
};

template <class R>
__device__ __forceinline__ R div_corrected(R x, R rho, R y) {
    const R q0 = x * y;
    const R q1 = fmaR(fmaR(-q0, rho, x), y, q0);
    return copysign(fmaR(fmaR(-q1, rho, x), y, q1), x);
}

template <class R>
__device__ __forceinline__ bool rho_in_range(R rho) {
    return rho >= DivRange<R>::rlo && rho <= DivRange<R>::rhi;
}

// Whether the three numerators lie where div_corrected is exact.  In general
// each one is 0 or within [xlo, xhi].  XS: populations decoded from a 16-bit
// code (FP32 arithmetic).  Every value such a code decodes to is a multiple
// of the format's smallest magnitude (FP16 2^-24, FP16S 2^-24 before its
// 2^-15 scale, FP16C and the posits 2^-59 at the least) and FP32 sums of such
// multiples stay multiples, so a nonzero j_a 2^-SL is at least 2^-59 in
// magnitude; with k.xsafe the force adds a multiple of 2^-100 (|F_a| >= 2^-76)
// that keeps a nonzero x_a at or above 2^-100.  Only the upper bound is then
// open -- an FP16 code may decode to infinity -- and one comparison of the
// largest magnitude settles it.  A NaN numerator escapes the maximum, but
// gives a NaN quotient on both routes, which the clamp that follows maps to
// the same value.
template <class R, bool XS>
__device__ __forceinline__ bool numerators_ok(const Relax<R>& k, const R* x) {
    if constexpr (XS) {
        if (k.xsafe) return maxR(maxR(fabs(x[0]), fabs(x[1])), fabs(x[2])) <= DivRange<R>::xhi;
    }
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const R ax = fabs(x[a]);
        ok = ok && (x[a] == R(0) || (ax >= DivRange<R>::xlo && ax <= DivRange<R>::xhi));
    }
    return ok;
}

// the numerators x_a = j_a 2^-SL (+ F_a / 2); j is the scaled momentum and
// its 2^-SL exact
template <class R, int SL>
__device__ __forceinline__ void numerators(const Relax<R>& k, const R* j, R* x) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const R jj = SL == 0 ? j[a] : j[a] * R(Pow2<SL>::down);
        x[a] = k.force ? fmaR(R(0.5), k.F[a], jj) : jj;
    }
}

template <class R, int SL, bool XS = false>
__device__ __forceinline__ void velocity(const Relax<R>& k, R rho, const R* j, R* u) {
    R x[3];
    numerators<R, SL>(k, j, x);
    const R y = R(1) / rho;
    const bool ok = rho_in_range(rho) && numerators_ok<R, XS>(k, x);
#pragma unroll
    for (int a = 0; a < 3; ++a) u[a] = div_corrected(x[a], rho, y);
    if (!ok) {
#pragma unroll
        for (int a = 0; a < 3; ++a) u[a] = x[a] / rho;
    }
}

// the same for two cells, whose reciprocals and corrections overlap; one
// fallback for both
template <class R, int SL, bool XS = false>
__device__ __forceinline__ void velocity_pair(const Relax<R>& k, R ra, const R* ja, R* ua, R rb, const R* jb,
                                              R* ub) {
    R xa[3], xb[3];
    numerators<R, SL>(k, ja, xa);
    numerators<R, SL>(k, jb, xb);
    const R ya = R(1) / ra, yb = R(1) / rb;
    const bool ok = rho_in_range(ra) && rho_in_range(rb) && numerators_ok<R, XS>(k, xa) &&
                    numerators_ok<R, XS>(k, xb);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        ua[a] = div_corrected(xa[a], ra, ya);
        ub[a] = div_corrected(xb[a], rb, yb);
    }
    if (!ok) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            ua[a] = xa[a] / ra;
            ub[a] = xb[a] / rb;
        }
    }
}

// Shifted equilibrium with three FMAs per population (footnote of Sec. 2.2):
// f^eq-s = A (0.5 (B^2 + C) +- B) + D, A = w rho, B = 3 u.c, C = -3 u.u, D = w (rho - 1),
// returned times 2^SL (the weights carry the scale).  Bp receives B of the
// first member of every pair.  With sh = 0, D = w rho: the unshifted f^eq.
template <class V, class R, int SL>
__device__ __forceinline__ void equilibrium(R rho, const R* u, R* feq, R* Bp, R sh) {
    R t = u[0] * u[0];
    t = t + u[1] * u[1];
    if constexpr (V::D == 3) t = t + u[2] * u[2];
    const R C = R(-3) * t;
    const R u3[3] = {R(3) * u[0], R(3) * u[1], R(3) * u[2]};
    const R rhom1 = rho - sh;
    const R w0 = R(V::w(0) * Pow2<SL>::up);
    feq[0] = fmaR(w0 * rho, R(0.5) * C, w0 * rhom1);
    static_for<0, (V::Q - 1) / 2>([&](auto K) {
        constexpr int p = 2 * K.value + 1;
        const R w = R(V::w(p) * Pow2<SL>::up);
        const R A = w * rho, D = w * rhom1;
        const R B = csum<V, p, R>(u3);
        const R X = fmaR(B, B, C);
        feq[p] = fmaR(A, fmaR(R(0.5), X, B), D);
        feq[p + 1] = fmaR(A, fmaR(R(0.5), X, -B), D);
        Bp[p] = B;
    });
}

// Guo source S_i = 3 w_i ((c_i.F - u.F) + B_i (c_i.F)) with B_i = 3 c_i.u, times 2^SL
template <class V, class R, int SL>
__device__ __forceinline__ void guo_source(const Relax<R>& k, const R* u, const R* Bp, R* S) {
    R uF = u[0] * k.F[0];
    uF = fmaR(u[1], k.F[1], uF);
    if constexpr (V::D == 3) uF = fmaR(u[2], k.F[2], uF);
    S[0] = R(3.0 * V::w(0) * Pow2<SL>::up) * (-uF);
    static_for<0, (V::Q - 1) / 2>([&](auto K) {
        constexpr int p = 2 * K.value + 1;
        const R cF = csum<V, p, R>(k.F);
        const R w3 = R(3.0 * V::w(p) * Pow2<SL>::up);
        S[p] = w3 * fmaR(Bp[p], cF, cF - uF);
        S[p + 1] = w3 * fmaR(Bp[p], cF, (-cF) - uF);
    });
}

// streamed populations g -> post-collision populations (in place), both
// 2^SL f, given the density and the clamped velocity
template <class V, int COLL, class R, int SL>
__device__ __forceinline__ void collide_post(const Relax<R>& k, R* f, R rho, const R* u) {
    R feq[V::Q], Bp[V::Q], S[V::Q];
    equilibrium<V, R, SL>(rho, u, feq, Bp, k.sh);
    if (k.force) guo_source<V, R, SL>(k, u, Bp, S);
    if constexpr (COLL == 2) {   // MRT (D3Q19): f - M^-1 S M (f - f^eq) [+ M^-1 (I - S/2) M S_guo]
        static_assert(V::Q == 19, "MRT is defined for D3Q19");
        // fixed order: sums over the non-zero M_ki in index order from +0
        R d[19], n[19], t[19];
        static_for<0, 19>([&](auto I) { d[I.value] = f[I.value] - feq[I.value]; });
        static_for<0, 19>([&](auto K) {
            constexpr int kk = K.value;
            R m = R(0), sm = R(0);
            static_for<0, 19>([&](auto I) {
                constexpr int e = mrt_m<V>(kk, I.value);
                if constexpr (e != 0) {
                    m = fmaR(R(e), d[I.value], m);
                    if (k.force) sm = fmaR(R(e), S[I.value], sm);
                }
            });
            n[kk] = m * k.mrt_r[kk];
            t[kk] = k.force ? sm * k.mrt_p[kk] : R(0);
        });
        static_for<0, 19>([&](auto I) {
            constexpr int i = I.value;
            R acc = R(0), acc2 = R(0);
            static_for<0, 19>([&](auto K) {
                constexpr int e = mrt_m<V>(K.value, i);
                if constexpr (e != 0) {
                    acc = fmaR(R(e), n[K.value], acc);
                    if (k.force) acc2 = fmaR(R(e), t[K.value], acc2);
                }
            });
            f[i] = k.force ? (f[i] - acc) + acc2 : f[i] - acc;
        });
    } else if constexpr (COLL == 0) {   // SRT: fma(1 - omega, f, omega f^eq)
        if (k.force) {
            static_for<0, V::Q>([&](auto I) {
                constexpr int i = I.value;
                f[i] = fmaR(k.c1, f[i], fmaR(k.om, feq[i], k.cSp * S[i]));
            });
        } else {
            static_for<0, V::Q>([&](auto I) {
                constexpr int i = I.value;
                f[i] = fmaR(k.c1, f[i], k.om * feq[i]);
            });
        }
    } else {                     // TRT on the symmetric / antisymmetric parts of each pair
        const R a0 = f[0] - feq[0];
        f[0] = fmaR(-k.omp, a0, k.force ? fmaR(k.cSp, S[0], f[0]) : f[0]);
        static_for<0, (V::Q - 1) / 2>([&](auto K) {
            constexpr int p = 2 * K.value + 1, q = p + 1;
            // parts (a + b)/2 and (a - b)/2 relaxed with omega+ and omega-,
            // the halves carried by the rates (one product, exact halving)
            const R a = f[p] - feq[p], b = f[q] - feq[q];
            const R s = a + b, d = a - b;
            R fp = f[p], fq = f[q];
            if (k.force) {
                const R Ss = S[p] + S[q], Sd = S[p] - S[q];
                fp = fp + fmaR(k.cSmh, Sd, k.cSph * Ss);
                fq = fq + fmaR(-k.cSmh, Sd, k.cSph * Ss);
            }
            f[p] = fmaR(-k.ommh, d, fmaR(-k.omph, s, fp));
            f[q] = fmaR(k.ommh, d, fmaR(-k.omph, s, fq));
        });
    }
}

// each component clamped to [-cs, cs] (the paper's core limits |u_a| to c_s)
template <class R>
__device__ __forceinline__ void clamp_u(const Relax<R>& k, R* u) {
#pragma unroll
    for (int a = 0; a < 3; ++a) u[a] = minR(maxR(u[a], -k.cs), k.cs);
}

// one stream-collide update: moments, velocity, clamp, equilibrium,
// collision; XS: populations decoded from 16-bit codes (see numerators_ok)
template <class V, int COLL, class R, int SL, bool XS = false>
__device__ __forceinline__ void collide(const Relax<R>& k, R* f) {
    R rho, j[3], u[3];
    moments<V, R, SL>(f, rho, j, k.sh);
    velocity<R, SL, XS>(k, rho, j, u);
    clamp_u(k, u);
    collide_post<V, COLL, R, SL>(k, f, rho, u);
}

// two cells: the density and velocity of both first, so that their
// dependent chains (sums, reciprocal, corrections) overlap, then each cell's
// equilibrium and collision; the same values as two collide() calls
template <class V, int COLL, class R, int SL, bool XS = false>
__device__ __forceinline__ void collide_pair(const Relax<R>& k, R* fa, R* fb) {
    R ra, rb, ja[3], jb[3], ua[3], ub[3];
    moments<V, R, SL>(fa, ra, ja, k.sh);
    moments<V, R, SL>(fb, rb, jb, k.sh);
    velocity_pair<R, SL, XS>(k, ra, ja, ua, rb, jb, ub);
    clamp_u(k, ua);
    clamp_u(k, ub);
    collide_post<V, COLL, R, SL>(k, fa, ra, ua);
    collide_post<V, COLL, R, SL>(k, fb, rb, ub);
}

template <class V, class R, int SL>
__device__ __forceinline__ void equilibrium_only(R rho, const R* u, R* feq, R sh) {
    R Bp[V::Q];
    equilibrium<V, R, SL>(rho, u, feq, Bp, sh);
}

}  // namespace lbm
