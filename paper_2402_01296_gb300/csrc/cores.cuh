// Kernels built on the register-resident NTT core: the batched NTT, the
// tensor-square core and the fused key-switching core.
#pragma once

#include "device_api.h"
#include "ntt_core.cuh"

namespace bcn {

template <int LOGN, int R>
__global__ void __launch_bounds__((1 << LOGN) / R) k_ntt_fwd(uint32_t *__restrict__ data, PrimeMap pm,
                                                            const PrimeConst *__restrict__ pc,
                                                            const uint2 *__restrict__ tw) {
    using C = NttCore<LOGN, R>;
    extern __shared__ __align__(16) uint32_t sm[];
    const int limb = blockIdx.x, tid = threadIdx.x;
    const int p = prime_of(pm, limb);
    const uint32_t q = pc[p].q;
    uint32_t *a = data + (size_t)limb * C::N;
    uint32_t x[R];
    C::load_natural(x, a, tid);
    C::forward(x, sm, tid, q, tw + (size_t)p * C::N);
    C::store_ntt(x, a, tid);
}

template <int LOGN, int R>
__global__ void __launch_bounds__((1 << LOGN) / R) k_ntt_inv(uint32_t *__restrict__ data, PrimeMap pm,
                                                            const PrimeConst *__restrict__ pc,
                                                            const uint2 *__restrict__ tw) {
    using C = NttCore<LOGN, R>;
    extern __shared__ __align__(16) uint32_t sm[];
    const int limb = blockIdx.x, tid = threadIdx.x;
    const int p = prime_of(pm, limb);
    const PrimeConst P = pc[p];
    uint32_t *a = data + (size_t)limb * C::N;
    uint32_t x[R];
    C::load_ntt(x, a, tid);
    C::inverse(x, sm, tid, P.q, tw + (size_t)p * C::N, P.ninv, P.ninv_shoup);
    C::store_natural(x, a, tid);
}

// The lazy butterflies' additions selected by each kernel's FMA bits go
// through the FMA pipe (ModQ::one read at run time) in blocks of at most 512
// threads (128 registers); in the 1024-thread blocks of the N = 16384 square
// kernel the compile-time 1 folds them back into plain additions.
template <int LOGN, int R>
constexpr bool kFmaOne = (1 << LOGN) / R <= 512;

// Lazy-butterfly additions on the FMA pipe, per kernel (measured at N = 8192:
// the square kernel's transforms are best with only the forward min's
// subtraction there, the key switch's with the inverse min's as well; its
// running sums add on the ALU pipe)
#ifndef BCN_FMA_SQ
#define BCN_FMA_SQ kFmaFwdMin
#endif
#ifndef BCN_FMA_KS
#define BCN_FMA_KS (kFmaFwdMin | kFmaInvMin)
#endif
constexpr int kFmaSquare = BCN_FMA_SQ, kFmaKs = BCN_FMA_KS;

// Pairs of independent transforms run in lockstep (shared twiddle loads and
// barriers, twice the independent work per thread) where the registers allow
// it: up to N = 8192.
template <int LOGN, int R>
constexpr bool kDual = (1 << LOGN) / R <= 512 && R <= 16;

// Register budget per thread of the fused kernels (sets their blocks per SM).
#ifndef BCN_CORE_REGS
#define BCN_CORE_REGS 128
#endif
template <int T>
struct CoreOcc {
    static constexpr int B = 65536 / (T * BCN_CORE_REGS);
    static constexpr int MIN_BLOCKS = B > 32 ? 32 : (B < 1 ? 1 : B);
};

// Square activation, first half: forward NTT of c0 and c1 of one limb,
// tensor square (c0^2, 2 c0 c1, c1^2) in the NTT domain, inverse NTT of the
// three products.  Y [C][2][n][N] -> D [C][3][n][N], coefficient form; with
// D2N != nullptr also c1^2 in the NTT domain (last-pass layout of the NTT) to
// D2N [C][n][N], which the key-switching kernel reuses on the digit's own prime.
// The products are formed with R*N^{-1} in place of R, so they carry the
// inverse transform's N^{-1} already.  grid (n, C): one block per (limb, ct).
template <int LOGN, int R>
__global__ void __launch_bounds__((1 << LOGN) / R, CoreOcc<(1 << LOGN) / R>::MIN_BLOCKS)
    k_square_core(const uint32_t *__restrict__ Y, uint32_t *__restrict__ D, uint32_t *__restrict__ D2N, int n,
                  const PrimeConst *__restrict__ pc, const uint2 *__restrict__ twf, const uint2 *__restrict__ twi) {
    using C = NttCore<LOGN, R, true, kFmaSquare>;  // data primes only (q < 2^30): lazy butterflies
    constexpr int N = C::N, T = C::T;
    extern __shared__ __align__(16) uint32_t sm[];
    const int i = blockIdx.x, ct = blockIdx.y, tid = threadIdx.x;
    const PrimeConst P = pc[i];
    const uint2 *tf = twf + (size_t)i * N, *ti = twi + (size_t)i * N;
    if constexpr (kDual<LOGN, R>) {
        // c0 and c1 transformed together (two exchange buffers), then d0 and d1
        // back together; d2 waits in a thread-private parking area (u*T + tid)
        uint32_t *s2 = sm + 2 * C::SMEM_WORDS;
        const ModQ mq(P.q, kFmaOne<LOGN, R> ? P.one : 1u);
        uint32_t x[2][R];
        C::load_natural(x[0], Y + (((size_t)ct * 2 + 0) * n + i) * N, tid);
        C::load_natural(x[1], Y + (((size_t)ct * 2 + 1) * n + i) * N, tid);
        C::forward_n(x, sm, tid, mq, tf);
        uint32_t *d2n = D2N != nullptr ? D2N + ((size_t)ct * n + i) * N : nullptr;
        constexpr int V = C::NTT_QUADS ? 4 : (C::NTT_PAIRS ? 2 : 1);
#pragma unroll
        for (int u0 = 0; u0 < R; u0 += V) {
            uint32_t c2[V];  // c1^2, canonical, for the key switch's own-digit term
#pragma unroll
            for (int z = 0; z < V; z++) {
                const int u = u0 + z;
                const uint32_t a = x[0][u], b = x[1][u];  // [0, 4q)
                c2[z] = mont_mul(shoup_mul(b, P.r_mod, P.r_shoup, P.q), b, P.q, P.qneg_inv);
                const uint32_t aRN = shoup_mul(a, P.rn, P.rn_shoup, P.q);
                const uint32_t bRN = shoup_mul(b, P.rn, P.rn_shoup, P.q);
                const uint32_t ab = mont_mul(aRN, b, P.q, P.qneg_inv);
                x[0][u] = mont_mul(aRN, a, P.q, P.qneg_inv);  // c0^2 / N
                x[1][u] = add_mod(ab, ab, P.q);                // 2 c0 c1 / N
                s2[u * T + tid] = mont_mul(bRN, b, P.q, P.qneg_inv);  // c1^2 / N
            }
            if (d2n != nullptr) {
                const int e = C::ntt_elem(u0, tid);
                if constexpr (V == 4)
                    *reinterpret_cast<uint4 *>(d2n + e) = make_uint4(c2[0], c2[1], c2[2], c2[3]);
                else if constexpr (V == 2)
                    *reinterpret_cast<uint2 *>(d2n + e) = make_uint2(c2[0], c2[1]);
                else
                    d2n[e] = c2[0];
            }
        }
        C::inverse_unscaled_n(x, sm, tid, mq, ti);
        C::store_natural(x[0], D + (((size_t)ct * 3 + 0) * n + i) * N, tid);
        C::store_natural(x[1], D + (((size_t)ct * 3 + 1) * n + i) * N, tid);
#pragma unroll
        for (int u = 0; u < R; u++) x[0][u] = s2[u * T + tid];
        C::inverse_unscaled(x[0], sm, tid, mq, ti);
        C::store_natural(x[0], D + (((size_t)ct * 3 + 2) * n + i) * N, tid);
        return;
    }
    // exchange buffer, then two thread-private parking areas (slot u*T + tid)
    uint32_t *s1 = sm + C::SMEM_WORDS, *s2 = s1 + N;
    uint32_t x[R];
    // c0 -> NTT, parked in s1
    C::load_natural(x, Y + (((size_t)ct * 2 + 0) * n + i) * N, tid);
    C::forward(x, sm, tid, ModQ(P.q, kFmaOne<LOGN, R> ? P.one : 1u), tf);
#pragma unroll
    for (int u = 0; u < R; u++) s1[u * T + tid] = x[u];
    // c1 -> NTT; c0^2/N in registers, 2 c0 c1/N in s1, c1^2/N in s2 (inputs in [0, 4q))
    C::load_natural(x, Y + (((size_t)ct * 2 + 1) * n + i) * N, tid);
    C::forward(x, sm, tid, ModQ(P.q, kFmaOne<LOGN, R> ? P.one : 1u), tf);
    if (D2N != nullptr) {
        uint32_t y[R];
#pragma unroll
        for (int u = 0; u < R; u++) {
            const uint32_t bR = shoup_mul(x[u], P.r_mod, P.r_shoup, P.q);
            y[u] = mont_mul(bR, x[u], P.q, P.qneg_inv);  // c1^2, canonical
        }
        C::store_ntt(y, D2N + ((size_t)ct * n + i) * N, tid);
    }
#pragma unroll
    for (int u = 0; u < R; u++) {
        const uint32_t a = s1[u * T + tid], b = x[u];
        const uint32_t aRN = shoup_mul(a, P.rn, P.rn_shoup, P.q);
        const uint32_t bRN = shoup_mul(b, P.rn, P.rn_shoup, P.q);
        const uint32_t ab = mont_mul(aRN, b, P.q, P.qneg_inv);
        s1[u * T + tid] = add_mod(ab, ab, P.q);
        s2[u * T + tid] = mont_mul(bRN, b, P.q, P.qneg_inv);
        x[u] = mont_mul(aRN, a, P.q, P.qneg_inv);
    }
    C::inverse_unscaled(x, sm, tid, ModQ(P.q, kFmaOne<LOGN, R> ? P.one : 1u), ti);
    C::store_natural(x, D + (((size_t)ct * 3 + 0) * n + i) * N, tid);
#pragma unroll
    for (int u = 0; u < R; u++) x[u] = s1[u * T + tid];
    C::inverse_unscaled(x, sm, tid, ModQ(P.q, kFmaOne<LOGN, R> ? P.one : 1u), ti);
    C::store_natural(x, D + (((size_t)ct * 3 + 1) * n + i) * N, tid);
#pragma unroll
    for (int u = 0; u < R; u++) x[u] = s2[u * T + tid];
    C::inverse_unscaled(x, sm, tid, ModQ(P.q, kFmaOne<LOGN, R> ? P.one : 1u), ti);
    C::store_natural(x, D + (((size_t)ct * 3 + 2) * n + i) * N, tid);
}

// Key switching of d2, fused per (target prime t, ciphertext): for every
// digit j, ModUp of d2 into prime t (the residue itself on the digit's own
// primes -- taken from D2N in the NTT domain when given -- else the centred
// fast basis conversion
//     sum_u r_u * Dhat_u - #{u : r_u > (q_u-1)/2} * D_j,  r_u = [x_u Dhat_u^{-1}]_{q_u},
// which for one-prime digits is d mod t, less q_j mod t when d > (q_j-1)/2),
// forward NTT, and the product with evk_j (prepared as k*R*N^{-1}, so one
// Montgomery product gives k*x/N) accumulated for both key halves; then the
// inverse NTT of the two sums.  No extended-basis limb is stored.
// D [C][3][n][N] (d2 in coefficient form) -> ACC [C][2][n+K][N] (coefficient form).
template <int LOGN, int R, bool LAZY>
__device__ __forceinline__ void ks_core_body(const uint32_t *__restrict__ D, const uint32_t *__restrict__ D2N,
                                             const uint32_t *__restrict__ evk, uint32_t *__restrict__ acc_out,
                                             int n, const KsDev &ks, const PrimeConst *__restrict__ pc,
                                             const uint2 *__restrict__ twf, const uint2 *__restrict__ twi) {
    using C = NttCore<LOGN, R, LAZY, kFmaKs>;
    constexpr int N = C::N, T = C::T;
    // running sums r0 += x k0 / R, r1 += x k1 / R: kept in [0, 2q) with lazy
    // Montgomery products on the data primes (the lazy inverse NTT takes
    // [0, 2q)), canonical on the special primes
    // (additions through the FMA pipe as in the lazy butterflies)
    auto ks_accumulate = [](uint32_t &r0, uint32_t &r1, uint32_t xv, uint32_t w0, uint32_t w1,
                            const PrimeConst &P) {
        if constexpr (LAZY) {
            const uint32_t nq2 = 0u - 2 * P.q;
            const uint32_t a0 = mont_mul_lazy(xv, w0, P.q, P.qneg_inv) + r0;
            const uint32_t a1 = mont_mul_lazy(xv, w1, P.q, P.qneg_inv) + r1;
            r0 = min(a0, a0 + nq2);
            r1 = min(a1, a1 + nq2);
        } else {
            r0 = add_mod(r0, mont_mul(xv, w0, P.q, P.qneg_inv), P.q);
            r1 = add_mod(r1, mont_mul(xv, w1, P.q, P.qneg_inv), P.q);
        }
    };
    extern __shared__ __align__(16) uint32_t sm[];
    // exchange buffer(s) -- two where the final inverse transforms run together --
    // then the two running sums in thread-private slots u*T + tid
    uint32_t *s0 = sm + (kDual<LOGN, R> ? 2 : 1) * C::SMEM_WORDS, *s1 = s0 + N;
    const int t = blockIdx.x, ct = blockIdx.y, tid = threadIdx.x;
    const int A = ks.alpha, dnum = (n + A - 1) / A, nb = n + ks.K;
    const int pt = t < n ? t : ks.L + (t - n);
    const PrimeConst P = pc[pt];
    const uint2 *tf = twf + (size_t)pt * N, *ti = twi + (size_t)pt * N;
    const uint32_t *x2 = D + ((size_t)ct * 3 + 2) * n * N;
    // product of a digit's NTT-domain ModUp limb with both halves of its key,
    // added to the running sums
    auto key_product = [&](const uint32_t(&xr)[R], int j) {
        const uint32_t *k0 = evk + ((size_t)(j * 2 + 0) * ks.P + pt) * N;
        const uint32_t *k1 = evk + ((size_t)(j * 2 + 1) * ks.P + pt) * N;
        if constexpr (C::NTT_QUADS) {
#pragma unroll
            for (int u = 0; u < R; u += 4) {
                const int e = C::ntt_elem(u, tid);
                const uint4 v0 = __ldg(reinterpret_cast<const uint4 *>(k0 + e));
                const uint4 v1 = __ldg(reinterpret_cast<const uint4 *>(k1 + e));
                const uint32_t w0[4] = {v0.x, v0.y, v0.z, v0.w}, w1[4] = {v1.x, v1.y, v1.z, v1.w};
#pragma unroll
                for (int z = 0; z < 4; z++) ks_accumulate(s0[(u + z) * T + tid], s1[(u + z) * T + tid], xr[u + z],
                                                          w0[z], w1[z], P);
            }
        } else if constexpr (C::NTT_PAIRS) {
#pragma unroll
            for (int u = 0; u < R; u += 2) {
                const int e = C::ntt_elem(u, tid);
                const uint2 v0 = __ldg(reinterpret_cast<const uint2 *>(k0 + e));
                const uint2 v1 = __ldg(reinterpret_cast<const uint2 *>(k1 + e));
                const uint32_t w0[2] = {v0.x, v0.y}, w1[2] = {v1.x, v1.y};
#pragma unroll
                for (int z = 0; z < 2; z++) ks_accumulate(s0[(u + z) * T + tid], s1[(u + z) * T + tid], xr[u + z],
                                                          w0[z], w1[z], P);
            }
        } else {
#pragma unroll
            for (int u = 0; u < R; u++) {
                const int e = C::ntt_elem(u, tid);
                ks_accumulate(s0[u * T + tid], s1[u * T + tid], xr[u], __ldg(k0 + e), __ldg(k1 + e), P);
            }
        }
    };
    // the same for two digits' limbs, one pass over the sums
    auto key_product2 = [&](const uint32_t(&xr)[2][R], int ja, int jb) {
        const uint32_t *ka0 = evk + ((size_t)(ja * 2 + 0) * ks.P + pt) * N;
        const uint32_t *ka1 = evk + ((size_t)(ja * 2 + 1) * ks.P + pt) * N;
        const uint32_t *kb0 = evk + ((size_t)(jb * 2 + 0) * ks.P + pt) * N;
        const uint32_t *kb1 = evk + ((size_t)(jb * 2 + 1) * ks.P + pt) * N;
        static_assert(C::NTT_QUADS || C::NTT_PAIRS, "paired key products read whole pairs");
        constexpr int V = C::NTT_QUADS ? 4 : 2;
#pragma unroll
        for (int u = 0; u < R; u += V) {
            const int e = C::ntt_elem(u, tid);
            uint32_t wa0[V], wa1[V], wb0[V], wb1[V];
            if constexpr (V == 4) {
                *reinterpret_cast<uint4 *>(wa0) = __ldg(reinterpret_cast<const uint4 *>(ka0 + e));
                *reinterpret_cast<uint4 *>(wa1) = __ldg(reinterpret_cast<const uint4 *>(ka1 + e));
                *reinterpret_cast<uint4 *>(wb0) = __ldg(reinterpret_cast<const uint4 *>(kb0 + e));
                *reinterpret_cast<uint4 *>(wb1) = __ldg(reinterpret_cast<const uint4 *>(kb1 + e));
            } else {
                *reinterpret_cast<uint2 *>(wa0) = __ldg(reinterpret_cast<const uint2 *>(ka0 + e));
                *reinterpret_cast<uint2 *>(wa1) = __ldg(reinterpret_cast<const uint2 *>(ka1 + e));
                *reinterpret_cast<uint2 *>(wb0) = __ldg(reinterpret_cast<const uint2 *>(kb0 + e));
                *reinterpret_cast<uint2 *>(wb1) = __ldg(reinterpret_cast<const uint2 *>(kb1 + e));
            }
#pragma unroll
            for (int z = 0; z < V; z++) {
                uint32_t r0 = s0[(u + z) * T + tid], r1 = s1[(u + z) * T + tid];
                ks_accumulate(r0, r1, xr[0][u + z], wa0[z], wa1[z], P);
                ks_accumulate(r0, r1, xr[1][u + z], wb0[z], wb1[z], P);
                s0[(u + z) * T + tid] = r0;
                s1[(u + z) * T + tid] = r1;
            }
        }
    };
    uint32_t x[R];
#pragma unroll
    for (int u = 0; u < R; u++) s0[u * T + tid] = s1[u * T + tid] = 0;
    bool summed = false;
    if constexpr (LAZY && kDual<LOGN, R>) {
        if (A == 1) {
            // one-prime digits: the digit's own limb from D2N when given; the
            // others lifted (d, less q_j mod t when d > (q_j-1)/2; the own
            // limb unchanged) and transformed two at a time in lockstep
            const bool own_ntt = t < n && D2N != nullptr;
            if (own_ntt) {
                C::load_ntt(x, D2N + ((size_t)ct * n + t) * N, tid);
                key_product(x, t);
            }
            auto lift = [&](uint32_t(&xr)[R], int j) {
                uint32_t half = 0xFFFFFFFFu, tmq = 0u;
                if (j != t) {
                    half = pc[j].half;
                    tmq = P.q - ks.dprod[(size_t)(n * ks.dnum_max + j) * ks.P + pt];  // t - (q_j mod t)
                }
                const uint32_t *xj = x2 + (size_t)j * N;
#pragma unroll
                for (int u = 0; u < R; u++) {
                    const uint32_t d = __ldg(xj + C::nat_elem(u, tid));
                    xr[u] = d + (d > half ? tmq : 0u);
                }
            };
            auto skip_own = [&](int j) { return own_ntt && j == t ? j + 1 : j; };
            uint32_t y[2][R];
            for (int j = skip_own(0); j < n;) {
                const int j1 = skip_own(j + 1);
                if (j1 < n) {
                    lift(y[0], j);
                    lift(y[1], j1);
                    C::template forward_n<2>(y, sm, tid, ModQ(P.q, kFmaOne<LOGN, R> ? P.one : 1u), tf);
                    key_product2(y, j, j1);
                    j = skip_own(j1 + 1);
                } else {
                    lift(x, j);
                    C::forward(x, sm, tid, ModQ(P.q, kFmaOne<LOGN, R> ? P.one : 1u), tf);
                    key_product(x, j);
                    j = n;
                }
            }
            summed = true;
        }
    }
    for (int j = 0; j < dnum && !summed; j++) {
        const int lo = j * A, hi = min(lo + A, n);
        if (t >= lo && t < hi && D2N != nullptr) {
            C::load_ntt(x, D2N + ((size_t)ct * n + t) * N, tid);
        } else {
            if (t >= lo && t < hi) {
                C::load_natural(x, x2 + (size_t)t * N, tid);
            } else if (A == 1) {
                const uint32_t half = pc[j].half;
                const uint32_t dp = ks.dprod[(size_t)(n * ks.dnum_max + j) * ks.P + pt];  // q_j mod t
                const uint32_t *xj = x2 + (size_t)j * N;
                if constexpr (LAZY) {
                    // d - [d > (q_j-1)/2] q_j as d + (t - q_j mod t): below q_j + t < 3t (the
                    // data primes are within a factor 2), a valid lazy NTT input
                    const uint32_t tmq = P.q - dp;
#pragma unroll
                    for (int u = 0; u < R; u++) {
                        const uint32_t d = __ldg(xj + C::nat_elem(u, tid));
                        x[u] = d + (d > half ? tmq : 0u);
                    }
                } else {
#pragma unroll
                    for (int u = 0; u < R; u++) {
                        const uint32_t d = __ldg(xj + C::nat_elem(u, tid));
                        uint32_t y = reduce_once(d, P.q);  // d < q_j < 2t
                        if (d > half) y = sub_mod(y, dp, P.q);
                        x[u] = y;
                    }
                }
            } else {
#pragma unroll
                for (int u = 0; u < R; u++) x[u] = 0;
                const uint32_t dp = ks.dprod[(size_t)(n * ks.dnum_max + j) * ks.P + pt];
                for (int v = 0; v < hi - lo; v++) {
                    const int i = lo + v;
                    const uint32_t qi = pc[i].q, half = pc[i].half;
                    const uint2 di = ks.dhat_inv[(size_t)(n * ks.dnum_max + j) * A + v];
                    const uint2 dh = ks.dhat[((size_t)(n * ks.dnum_max + j) * A + v) * ks.P + pt];
                    const uint32_t *xi = x2 + (size_t)i * N;
#pragma unroll
                    for (int u = 0; u < R; u++) {
                        const uint32_t r = shoup_mul(__ldg(xi + C::nat_elem(u, tid)), di.x, di.y, qi);
                        uint32_t y = add_mod(x[u], shoup_mul(r, dh.x, dh.y, P.q), P.q);
                        if (r > half) y = sub_mod(y, dp, P.q);
                        x[u] = y;
                    }
                }
            }
            C::forward(x, sm, tid, ModQ(P.q, kFmaOne<LOGN, R> ? P.one : 1u), tf);
        }
        key_product(x, j);
    }
    if constexpr (kDual<LOGN, R>) {
        uint32_t y[2][R];
#pragma unroll
        for (int u = 0; u < R; u++) {
            y[0][u] = s0[u * T + tid];
            y[1][u] = s1[u * T + tid];
        }
        C::inverse_unscaled_n(y, sm, tid, ModQ(P.q, kFmaOne<LOGN, R> ? P.one : 1u), ti);
        C::store_natural(y[0], acc_out + (((size_t)ct * 2 + 0) * nb + t) * N, tid);
        C::store_natural(y[1], acc_out + (((size_t)ct * 2 + 1) * nb + t) * N, tid);
        return;
    }
#pragma unroll
    for (int u = 0; u < R; u++) x[u] = s0[u * T + tid];
    C::inverse_unscaled(x, sm, tid, ModQ(P.q, kFmaOne<LOGN, R> ? P.one : 1u), ti);
    C::store_natural(x, acc_out + (((size_t)ct * 2 + 0) * nb + t) * N, tid);
#pragma unroll
    for (int u = 0; u < R; u++) x[u] = s1[u * T + tid];
    C::inverse_unscaled(x, sm, tid, ModQ(P.q, kFmaOne<LOGN, R> ? P.one : 1u), ti);
    C::store_natural(x, acc_out + (((size_t)ct * 2 + 1) * nb + t) * N, tid);
}

// grid (n+K, C); lazy butterflies for the data primes (< 2^30), strict ones for
// the special primes (< 2^31)
template <int LOGN, int R>
__global__ void __launch_bounds__((1 << LOGN) / R, CoreOcc<(1 << LOGN) / R>::MIN_BLOCKS)
    k_ks_core(const uint32_t *__restrict__ D, const uint32_t *__restrict__ D2N, const uint32_t *__restrict__ evk,
              uint32_t *__restrict__ acc_out, int n, KsDev ks, const PrimeConst *__restrict__ pc,
              const uint2 *__restrict__ twf, const uint2 *__restrict__ twi) {
    const int t = blockIdx.x;
    const int pt = t < n ? t : ks.L + (t - n);
    if (pc[pt].q < (1u << 30))
        ks_core_body<LOGN, R, true>(D, D2N, evk, acc_out, n, ks, pc, twf, twi);
    else
        ks_core_body<LOGN, R, false>(D, D2N, evk, acc_out, n, ks, pc, twf, twi);
}

// R residues per thread for the NTT and square kernels, RKS for the key switch
template <int LOGN, int R, int RKS = R>
struct CoreImpl {
    using Core = NttCore<LOGN, R>;
    using CoreKs = NttCore<LOGN, RKS>;
    static constexpr size_t SMEM = (size_t)Core::SMEM_WORDS * 4;            // NTT alone
    // NTT alone; + two parking areas (or a second exchange buffer and one)
    static constexpr size_t SMEM3 =
        ((size_t)(kDual<LOGN, R> ? 2 * Core::SMEM_WORDS + Core::N : Core::SMEM_WORDS + 2 * Core::N)) * 4;
    // key switch: exchange buffer(s) and the two running sums
    static constexpr size_t SMEM_KS = ((size_t)(kDual<LOGN, RKS> ? 2 : 1) * CoreKs::SMEM_WORDS + 2 * CoreKs::N) * 4;

    static bcn_status ntt(const bcn_ctx *c, uint32_t *data, size_t n_limbs, PrimeMap pm, bool inverse,
                          cudaStream_t st) {
        if (inverse)
            k_ntt_inv<LOGN, R><<<(unsigned)n_limbs, Core::T, SMEM, st>>>(data, pm, c->d_pc, c->d_tw_inv);
        else
            k_ntt_fwd<LOGN, R><<<(unsigned)n_limbs, Core::T, SMEM, st>>>(data, pm, c->d_pc, c->d_tw_fwd);
        return check_launch("NTT");
    }
    static bcn_status square(const bcn_ctx *c, int n, const uint32_t *Y, uint32_t *D, uint32_t *D2N, int C,
                             cudaStream_t st) {
        k_square_core<LOGN, R><<<dim3(n, C), Core::T, SMEM3, st>>>(Y, D, D2N, n, c->d_pc, c->d_tw_fwd,
                                                                   c->d_tw_inv);
        return check_launch("k_square_core");
    }
    static bcn_status keyswitch(const bcn_ctx *c, int n, const uint32_t *D, const uint32_t *D2N,
                                const uint32_t *evk, uint32_t *acc, int C, cudaStream_t st) {
        k_ks_core<LOGN, RKS><<<dim3(n + c->K, C), CoreKs::T, SMEM_KS, st>>>(D, D2N, evk, acc, n, ks_dev(c), c->d_pc,
                                                                     c->d_tw_fwd, c->d_tw_inv);
        return check_launch("k_ks_core");
    }
    static bcn_status setup() {
        const int smem = (int)SMEM, smem3 = (int)SMEM3, smem_ks = (int)SMEM_KS;
        if (cudaFuncSetAttribute(k_ntt_fwd<LOGN, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
                cudaSuccess ||
            cudaFuncSetAttribute(k_ntt_inv<LOGN, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
                cudaSuccess ||
            cudaFuncSetAttribute(k_square_core<LOGN, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem3) !=
                cudaSuccess ||
            cudaFuncSetAttribute(k_ks_core<LOGN, RKS>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_ks) !=
                cudaSuccess ||
            cudaFuncSetAttribute(k_square_core<LOGN, R>, cudaFuncAttributePreferredSharedMemoryCarveout, 100) !=
                cudaSuccess ||
            cudaFuncSetAttribute(k_ks_core<LOGN, RKS>, cudaFuncAttributePreferredSharedMemoryCarveout, 100) !=
                cudaSuccess)
            return fail(BCN_E_CUDA, "cudaFuncSetAttribute failed for the NTT-based kernels");
        return BCN_OK;
    }
    static const CoreFns *fns() {
        static const CoreFns f = {&ntt, &square, &keyswitch, &setup};
        return &f;
    }
};

}  // namespace bcn
