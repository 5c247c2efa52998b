// modarith.cuh -- 64-bit modular arithmetic on the integer pipes (sm_103a).
//
// Moduli are primes p < 2^60 (Sec. III-A-1). Products are built from
// __umul64hi and the low 64-bit product; no 128-bit type is used on the device.
//
//  * Shoup multiplication by a constant W with precomputed W' = floor(W 2^64/p)
//    (the W' of Algorithm 1): for any Y < 2^64, T = W Y - floor(W' Y / 2^64) p
//    lies in [0, 2p).
//  * Harvey's lazy forward butterfly (Algorithm 1): X, Y in [0, 4p) ->
//    X' = X + W Y, Y' = X - W Y (mod p), both in [0, 4p).
//  * The matching Gentleman-Sande inverse butterfly on [0, 2p).
//  * Barrett reduction of a 128-bit z < 2 p^2 (Barrett 1986; the mad_mod of
//    Sec. III-A-1 feeds it a0 b1 + a1 b0 and reduces once).
#pragma once
#include <stdint.h>

namespace he {

typedef uint64_t u64;
typedef uint32_t u32;

// Constants of one prime, resident in device memory.
struct PrimeConst {
    u64 p;
    u64 two_p;
    u64 four_p;
    u64 neg_p;       // 2^64 - p
    u64 mu;          // floor(2^(2b+2) / p), b = bit length of p
    u64 ninv;        // N^-1 mod p
    u64 ninv_sh;     // its Shoup quotient
    u64 w1ninv;      // psi^-brv(1) * N^-1 mod p (last inverse stage)
    u64 w1ninv_sh;
    u64 one_sh;      // floor(2^64 / p): the Shoup quotient of 1 (reduce_word)
    u32 bits;        // b
    u32 h4;          // ceil(4p / 2^32): high-word threshold of the lazy reduction
};

// x >= m ? x - m : x for x, m < 2^63 (every caller: moduli below 2^60 and
// values below 16p). The sign of x - m decides, which saves the 64-bit
// unsigned comparison (two compare instructions) of the plain form.
__device__ __forceinline__ u64 reduce_once(u64 x, u64 m)
{
    const u64 r = x - m;
    return (long long)r < 0 ? x : r;
}

__device__ __forceinline__ u64 add_mod(u64 a, u64 b, u64 p) { return reduce_once(a + b, p); }

// a - b mod p for a, b < p < 2^62, by the sign of a - b.
__device__ __forceinline__ u64 sub_mod(u64 a, u64 b, u64 p)
{
    const u64 r = a - b;
    return (long long)r < 0 ? r + p : r;
}

// W * Y mod p in [0, 2p) for any Y < 2^64 (Shoup).
__device__ __forceinline__ u64 mul_shoup_lazy(u64 y, u64 w, u64 w_sh, u64 p)
{
    return w * y - __umul64hi(w_sh, y) * p;
}

__device__ __forceinline__ u64 mul_shoup(u64 y, u64 w, u64 w_sh, u64 p)
{
    return reduce_once(mul_shoup_lazy(y, w, w_sh, p), p);
}

// Shoup quotient from three of the four 32 x 32 partial products of
// W' Y / 2^64: with W' = Wh 2^32 + Wl and Y = Yh 2^32 + Yl,
//   W' Y / 2^64 = Wh Yh + hi(Wh Yl) + hi(Wl Yh) + f,  0 <= f < 3,
// (f collects the two dropped low halves and Wl Yl / 2^64), so the result
// Q' satisfies Q - 2 <= Q' <= Q for the exact Q = floor(W' Y / 2^64).
__device__ __forceinline__ u64 shoup_quotient_approx(u64 w_sh, u64 y)
{
    const u32 wl = (u32)w_sh, wh = (u32)(w_sh >> 32);
    const u32 yl = (u32)y, yh = (u32)(y >> 32);
    const u64 s = (u64)__umulhi(wh, yl) + (u64)__umulhi(wl, yh);
    return (u64)wh * yh + s;
}

// W * Y mod p in [0, 4p) for any Y < 2^64 and p < 2^62: the exact Shoup
// remainder lies in [0, 2p) and the quotient may be short by up to 2, so the
// integer W Y - Q' p lies in [0, 4p) and equals its value mod 2^64, formed as
// W Y + Q' (2^64 - p) in one multiply-add chain.
__device__ __forceinline__ u64 mul_shoup_lazy4(u64 y, u64 w, u64 w_sh, u64 neg_p)
{
    return w * y + shoup_quotient_approx(w_sh, y) * neg_p;
}

// Any word x reduced mod p: mul_shoup_lazy4 with W = 1 (W' = floor(2^64 / p))
// gives x - Q' p in [0, 4p), five 32 x 32 products (1 Y needs none) and few
// registers; reduce_word_canon adds two conditional subtractions for [0, p).
// Cheaper than Barrett of a single word, and it kept the mod-up transforms
// (which reduce a 60-bit digit for a smaller target on every load) from
// spilling.
__device__ __forceinline__ u64 reduce_word(u64 x, const PrimeConst &c)
{
    return mul_shoup_lazy4(x, 1, c.one_sh, c.neg_p);
}

__device__ __forceinline__ u64 reduce_word_canon(u64 x, const PrimeConst &c)
{
    return reduce_once(reduce_once(reduce_word(x, c), c.two_p), c.p);
}

// W Y mod p in [0, 4p) as mul_shoup_lazy4, with the multiply-add chains
// written out on 32-bit halves: the quotient Q' = Wh Yh + hi(Wh Yl) +
// hi(Wl Yh) (three products), then T = lo64(W Y) + lo64(Q' (2^64 - p)) (six
// products, carries by mad.lo.cc / madc.hi).
__device__ __forceinline__ u64 mul_shoup_lazy4_asm(u64 y, u64 w, u64 w_sh, u64 neg_p)
{
    u32 tl, th;
    asm("{\n\t"
        ".reg .u32 a, b, ql, qh;\n\t"
        "mul.hi.u32 a, %3, %4;\n\t"          // hi(Wh' Yl)
        "mul.hi.u32 b, %2, %5;\n\t"          // hi(Wl' Yh)
        "add.cc.u32 ql, a, b;\n\t"
        "addc.u32 qh, 0, 0;\n\t"
        "mad.lo.cc.u32 ql, %3, %5, ql;\n\t"  // + Wh' Yh
        "madc.hi.u32 qh, %3, %5, qh;\n\t"
        "mul.lo.u32 %0, %6, %4;\n\t"         // lo64(W Y)
        "mul.hi.u32 %1, %6, %4;\n\t"
        "mad.lo.u32 %1, %6, %5, %1;\n\t"
        "mad.lo.u32 %1, %7, %4, %1;\n\t"
        "mad.lo.cc.u32 %0, ql, %8, %0;\n\t"  // + lo64(Q' (2^64 - p))
        "madc.hi.u32 %1, ql, %8, %1;\n\t"
        "mad.lo.u32 %1, ql, %9, %1;\n\t"
        "mad.lo.u32 %1, qh, %8, %1;\n\t"
        "}"
        : "=&r"(tl), "=&r"(th)
        : "r"((u32)w_sh), "r"((u32)(w_sh >> 32)), "r"((u32)y), "r"((u32)(y >> 32)), "r"((u32)w),
          "r"((u32)(w >> 32)), "r"((u32)neg_p), "r"((u32)(neg_p >> 32)));
    return ((u64)th << 32) | tl;
}

// Forward butterfly (Harvey's, Algorithm 1, with wider lazy ranges): for
// 2^30 <= p < 2^60 and x, y in [0, 8p + 2^32),
//   x' = x + W y, y' = x - W y (mod p), both again in [0, 8p + 2^32).
// The reduction of x tests the high word only: if hi(x) >= ceil(4p / 2^32)
// then x >= 4p and x - 4p < 4p + 2^32; otherwise x < 4p + 2^32 already. With
// T = W y mod p in [0, 4p): x' < 8p + 2^32 and 0 < y' = x - T + 4p < 8p + 2^32.
// (8p + 2^32 < 2^64, so every value fits a word.)
__device__ __forceinline__ void ct_butterfly(u64 &x, u64 &y, u64 w, u64 w_sh, const PrimeConst &c)
{
    u64 X = x;
    if ((u32)(X >> 32) >= c.h4) X -= c.four_p;
#ifdef HE_BUTTERFLY_CXX
    const u64 T = mul_shoup_lazy4(y, w, w_sh, c.neg_p);
#else
    const u64 T = mul_shoup_lazy4_asm(y, w, w_sh, c.neg_p);
#endif
    x = X + T;
    y = X + c.four_p - T;
}

// [0, 8p + 2^32) -> [0, p) for p >= 2^30 (then 8p + 2^32 <= 12p < 16p):
// conditional subtractions of 8p, 4p, 2p and p. (A quotient estimate from the
// high word needs fewer instructions but measured slower here.)
__device__ __forceinline__ u64 reduce_from_fwd_range(u64 x, const PrimeConst &c)
{
    x = reduce_once(x, c.four_p << 1);
    x = reduce_once(x, c.four_p);
    x = reduce_once(x, c.two_p);
    return reduce_once(x, c.p);
}

// Last forward stage with canonical outputs: for x, y in [0, 8p + 2^32),
// x' = x + W y mod p and y' = x - W y mod p, both in [0, p). x goes to
// [0, p) by the four conditional subtractions above and T = W y mod p from
// [0, 4p) by two; the sum then needs one more and the difference a
// sign-tested correction (eight conditional steps for the pair, against four
// for each of the two lazy outputs).
__device__ __forceinline__ void ct_butterfly_canon(u64 &x, u64 &y, u64 w, u64 w_sh, const PrimeConst &c)
{
#ifdef HE_BUTTERFLY_CXX
    u64 T = mul_shoup_lazy4(y, w, w_sh, c.neg_p);
#else
    u64 T = mul_shoup_lazy4_asm(y, w, w_sh, c.neg_p);
#endif
    const u64 X = reduce_from_fwd_range(x, c);
    T = reduce_once(reduce_once(T, c.two_p), c.p);
    x = reduce_once(X + T, c.p);
    y = sub_mod(X, T, c.p);
}


// Inverse (Gentleman-Sande) butterfly on [0, 4p):
// x, y -> x + y, (x - y) W^-1 (mod p), both in [0, 4p): x + y < 8p reduces
// exactly once by 4p; x - y + 4p lies in (0, 8p) and its lazy Shoup product
// in [0, 4p).
__device__ __forceinline__ void gs_butterfly(u64 &x, u64 &y, u64 w, u64 w_sh, const PrimeConst &c)
{
    const u64 X = reduce_once(x + y, c.four_p);
    const u64 T = x - y + c.four_p;
#ifdef HE_BUTTERFLY_CXX
    y = mul_shoup_lazy4(T, w, w_sh, c.neg_p);
#else
    y = mul_shoup_lazy4_asm(T, w, w_sh, c.neg_p);
#endif
    x = X;
}

// 128-bit product as (hi, lo).
__device__ __forceinline__ void mul_wide(u64 a, u64 b, u64 &hi, u64 &lo)
{
    lo = a * b;
    hi = __umul64hi(a, b);
}

// Barrett reduction of z = (hi, lo) < 2 p^2 with p of b bits (3 <= b <= 60),
// mu = floor(2^(2b+2) / p). With q1 = floor(z / 2^(b-2)) and
// q3 = floor(q1 mu / 2^(b+4)): z/p - q3 < 2^(b-2)/p + q1/2^(b+4) + 1 < 2,
// so z - q3 p lies in [0, 2p) and one conditional subtraction finishes.
// q1 < 2^(b+3) and mu < 2^(b+3) fit one word each.
__device__ __forceinline__ u64 barrett_reduce(u64 hi, u64 lo, u64 p, u64 mu, u32 b)
{
    const u32 s1 = b - 2;                        // 1 .. 58
    u64 q1 = (hi << (64 - s1)) | (lo >> s1);
    u64 phi, plo;
    mul_wide(q1, mu, phi, plo);
    const u32 s2 = b + 4;                        // 7 .. 64
    u64 q3 = (phi << (64 - s2)) | ((plo >> 1) >> (s2 - 1));
    if (s2 == 64) q3 = phi;
    u64 r = lo - q3 * p;
    return reduce_once(r, p);
}

__device__ __forceinline__ u64 mul_mod(u64 a, u64 b, const PrimeConst &c)
{
    u64 hi, lo;
    mul_wide(a, b, hi, lo);
    return barrett_reduce(hi, lo, c.p, c.mu, c.bits);
}

// mad_mod of Sec. III-A-1: a0 b1 + a1 b0 mod p with a single reduction
// (the 128-bit sum is below 2 p^2).
__device__ __forceinline__ u64 mad2_mod(u64 a0, u64 b1, u64 a1, u64 b0, const PrimeConst &c)
{
    u64 h0, l0, h1, l1;
    mul_wide(a0, b1, h0, l0);
    mul_wide(a1, b0, h1, l1);
    u64 lo = l0 + l1;
    u64 hi = h0 + h1 + (lo < l0 ? 1 : 0);
    return barrett_reduce(hi, lo, c.p, c.mu, c.bits);
}

}  // namespace he
