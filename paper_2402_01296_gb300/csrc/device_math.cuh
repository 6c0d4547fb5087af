// 32-bit modular arithmetic for primes q < 2^31 on the device.
//   - Shoup multiplication by a precomputed constant w (w' = floor(w 2^32 / q)),
//     as in Harvey, "Faster arithmetic for number-theoretic transforms" (2014).
//   - Montgomery multiplication with R = 2^32 (Montgomery 1985) for products of
//     two variables; one operand carries the factor R.
//   - Barrett reduction of a 64-bit value with mu = floor(2^64 / q) (Barrett 1986).
// All results are canonical in [0, q) unless a name says otherwise.
#pragma once

#include <cstdint>

#include "bcn_internal.h"

namespace bcn {

__device__ __forceinline__ uint32_t add_mod(uint32_t a, uint32_t b, uint32_t q) {
    uint32_t s = a + b;  // < 2q < 2^32
    return s >= q ? s - q : s;
}

__device__ __forceinline__ uint32_t sub_mod(uint32_t a, uint32_t b, uint32_t q) {
    uint32_t d = a - b;
    return a >= b ? d : d + q;
}

// a * w mod q for any a < 2^32, w < q, wp = floor(w * 2^32 / q)
__device__ __forceinline__ uint32_t shoup_mul(uint32_t a, uint32_t w, uint32_t wp, uint32_t q) {
    uint32_t hi = __umulhi(a, wp);
    uint32_t r = a * w - hi * q;  // in [0, 2q)
    return r >= q ? r - q : r;
}

// a * b * 2^-32 mod q for a, b < q (< 2^31)
__device__ __forceinline__ uint32_t mont_mul(uint32_t a, uint32_t b, uint32_t q, uint32_t qneg_inv) {
    uint64_t t = (uint64_t)a * b;
    uint32_t m = (uint32_t)t * qneg_inv;
    uint32_t u = (uint32_t)((t + (uint64_t)m * q) >> 32);  // < 2q
    return u >= q ? u - q : u;
}

// x mod q for any x < 2^64 (mu = floor(2^64 / q))
__device__ __forceinline__ uint32_t barrett_reduce64(uint64_t x, uint32_t q, uint64_t mu) {
    uint64_t qh = __umul64hi(x, mu);
    uint64_t r = x - qh * q;  // in [0, 2q)
    return (uint32_t)(r >= q ? r - q : r);
}

}  // namespace bcn
