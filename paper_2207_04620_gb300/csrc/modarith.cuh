// 64-bit modular arithmetic for the device, all primes q < 2^62.
//
// * Shoup's precomputed-quotient product (NTL): for a constant w with
//   w' = floor(w * 2^64 / q), y*w - umulhi(y, w')*q lies in [0, 2q) for any
//   64-bit y.
// * Montgomery reduction (Montgomery 1985) with R = 2^64: for x < 2^64,
//   x * R^-1 mod q = umulhi(m, q) + (x != 0), m = x * (-q^-1 mod 2^64),
//   followed by one conditional subtraction.
// * Harvey's lazy butterflies (Harvey 2014) keep NTT values in [0, 4q).
#pragma once
#include <cstdint>

namespace hx {

struct PrimeConst {
    uint64_t q;
    uint64_t mneg;     // -q^-1 mod 2^64 (Montgomery)
    uint64_t bar;      // floor(2^64 / q): Shoup companion of w = 1
    uint64_t r_mod;    // 2^64 mod q
    uint64_t r_mod_sh; // Shoup companion of r_mod
    uint64_t n_inv;    // N^-1 mod q
    uint64_t n_inv_sh;
    uint64_t n_inv_w1;     // N^-1 * psi^-brv(1) mod q: the last inverse stage's twiddle with N^-1 folded in
    uint64_t n_inv_w1_sh;
};

__device__ __forceinline__ uint64_t shoup_lazy(uint64_t y, uint64_t w, uint64_t wsh, uint64_t q)
{
    return y * w - __umul64hi(y, wsh) * q;
}

__device__ __forceinline__ uint64_t csub(uint64_t x, uint64_t q) { return x >= q ? x - q : x; }

__device__ __forceinline__ uint64_t shoup(uint64_t y, uint64_t w, uint64_t wsh, uint64_t q)
{
    return csub(shoup_lazy(y, w, wsh, q), q);
}

// y mod q for any 64-bit y
__device__ __forceinline__ uint64_t reduce64(uint64_t y, uint64_t q, uint64_t bar)
{
    return csub(y - __umul64hi(y, bar) * q, q);
}

// x * 2^-64 mod q for any 64-bit x
__device__ __forceinline__ uint64_t mont64(uint64_t x, uint64_t q, uint64_t mneg)
{
    uint64_t m = x * mneg;
    uint64_t t = __umul64hi(m, q) + (x != 0 ? 1u : 0u);
    return csub(t, q);
}

// (hi*2^64 + lo) * 2^-64 mod q = hi + lo*2^-64 (mod q), for any 128-bit value
__device__ __forceinline__ uint64_t mont128(uint64_t hi, uint64_t lo, const PrimeConst &p)
{
    return csub(reduce64(hi, p.q, p.bar) + mont64(lo, p.q, p.mneg), p.q);
}

// (hi*2^64 + lo) * 2^-64 mod q in one Montgomery step (REDC), valid for hi < 3q: a sum of fewer
// than 24 products of residues, since q < 2^61 keeps each product's high word below q/8.  The
// quotient step leaves t = hi + umulhi(m, q) + [lo != 0] < 4q, two conditional subtractions.
__device__ __forceinline__ uint64_t redc_few(uint64_t hi, uint64_t lo, const PrimeConst &p)
{
    const uint64_t m = lo * p.mneg;
    uint64_t t = hi + __umul64hi(m, p.q) + (lo != 0 ? 1u : 0u);
    if (t >= 2 * p.q) t -= 2 * p.q;
    return csub(t, p.q);
}

// products accumulated per output for which redc_few applies
constexpr int kRedcFewTerms = 23;

__device__ __forceinline__ uint64_t addmod(uint64_t a, uint64_t b, uint64_t q) { return csub(a + b, q); }
__device__ __forceinline__ uint64_t submod(uint64_t a, uint64_t b, uint64_t q) { return a >= b ? a - b : a + q - b; }

// 128-bit accumulator built from the two 64-bit halves of products
struct Acc128 {
    uint64_t lo = 0, hi = 0;
    __device__ __forceinline__ void mac(uint64_t a, uint64_t b)
    {
        uint64_t l = a * b;
        uint64_t h = __umul64hi(a, b);
        lo += l;
        hi += h + (lo < l ? 1u : 0u);
    }
};

// a*b mod q for two standard residues: Montgomery gives a*b*2^-64, the Shoup
// product with (2^64 mod q) restores the factor.
__device__ __forceinline__ uint64_t mulmod(uint64_t a, uint64_t b, const PrimeConst &p)
{
    uint64_t t = redc_few(__umul64hi(a, b), a * b, p);
    return shoup(t, p.r_mod, p.r_mod_sh, p.q);
}

} // namespace hx
