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

// x - m if x >= m else x, for x < 2m <= 2^32 (one subtraction and one unsigned min)
__device__ __forceinline__ uint32_t reduce_once(uint32_t x, uint32_t m) { return min(x, x - m); }

__device__ __forceinline__ uint32_t add_mod(uint32_t a, uint32_t b, uint32_t q) {
    return reduce_once(a + b, q);  // a + b < 2q <= 2^32
}

__device__ __forceinline__ uint32_t sub_mod(uint32_t a, uint32_t b, uint32_t q) {
    return reduce_once(a + q - b, q);  // a + q - b in (0, 2q)
}

// a * w mod q up to one q: result in [0, 2q), for any a < 2^32
__device__ __forceinline__ uint32_t shoup_mul_lazy(uint32_t a, uint32_t w, uint32_t wp, uint32_t q) {
    return a * w - __umulhi(a, wp) * q;
}

// a * w mod q for any a < 2^32, w < q, wp = floor(w * 2^32 / q)
__device__ __forceinline__ uint32_t shoup_mul(uint32_t a, uint32_t w, uint32_t wp, uint32_t q) {
    return reduce_once(shoup_mul_lazy(a, w, wp, q), q);
}

// a * b * 2^-32 mod q for a < 4q, b < q, q < 2^30; or a, b < q < 2^31
__device__ __forceinline__ uint32_t mont_mul(uint32_t a, uint32_t b, uint32_t q, uint32_t qneg_inv) {
    uint64_t t = (uint64_t)a * b;
    uint32_t m = (uint32_t)t * qneg_inv;
    uint32_t u = (uint32_t)((t + (uint64_t)m * q) >> 32);  // < 2q
    return reduce_once(u, q);
}

// a * b * 2^-32 mod q up to one q: result in [0, 2q), for a < 4q, b < q, q < 2^30
__device__ __forceinline__ uint32_t mont_mul_lazy(uint32_t a, uint32_t b, uint32_t q, uint32_t qneg_inv) {
    uint64_t t = (uint64_t)a * b;
    uint32_t m = (uint32_t)t * qneg_inv;
    return (uint32_t)((t + (uint64_t)m * q) >> 32);
}

// x mod q for any x < 2^64 (mu = floor(2^64 / q))
__device__ __forceinline__ uint32_t barrett_reduce64(uint64_t x, uint32_t q, uint64_t mu) {
    uint64_t qh = __umul64hi(x, mu);
    uint32_t r = (uint32_t)(x - qh * q);  // in [0, 2q)
    return reduce_once(r, q);
}

// L2 prefetch hint for the 32-bit words [0, n_words) of a row: one 128-byte
// line per thread, the block's nthreads threads striding over the row
__device__ __forceinline__ void prefetch_row_l2(const uint32_t *row, int n_words, int tid, int nthreads) {
    for (int w = tid * 32; w < n_words; w += nthreads * 32) asm volatile("prefetch.global.L2 [%0];" ::"l"(row + w));
}

// x mod q for x < 2^59 and a data prime 2^29 < q < 2^30, with 32-bit
// multiplies (mu = floor(2^64 / q) as for barrett_reduce64): the quotient
// estimate floor(floor(x / 2^29) floor(2^61 / q) / 2^32) is at most 2 below
// floor(x / q) (x / 2^61 < 1/4 and 2^29 / q < 1) and never above it, so
// x - estimate q lies in [0, 3q) and fits 32 bits
__device__ __forceinline__ uint32_t reduce59(uint64_t x, uint32_t q, uint64_t mu) {
    const uint32_t qe = __umulhi((uint32_t)(x >> 29), (uint32_t)(mu >> 3));
    uint32_t r = (uint32_t)x - qe * q;  // [0, 3q)
    r = min(r, r - 2 * q);              // [0, 2q)
    return reduce_once(r, q);
}

}  // namespace bcn
