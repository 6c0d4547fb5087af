// Kernels built on the register-resident NTT core: the batched NTT, the
// tensor-square core and the fused key-switching core.
#pragma once

#include "device_api.h"
#include "ntt_core.cuh"

namespace bcn {

// In-place NTT of limb blockIdx.x of group blockIdx.y (groups `stride` words
// apart): natural order <-> last-pass layout.
template <int LOGN, int R>
__global__ void __launch_bounds__((1 << LOGN) / R) k_ntt_fwd(uint32_t *__restrict__ data, PrimeMap pm,
                                                            size_t stride, const PrimeConst *__restrict__ pc,
                                                            const uint2 *__restrict__ tw) {
    using C = NttCore<LOGN, R>;
    extern __shared__ __align__(16) uint32_t sm[];
    const int limb = blockIdx.x, tid = threadIdx.x;
    const int p = prime_of(pm, limb);
    const uint32_t q = pc[p].q;
    uint32_t *a = data + blockIdx.y * stride + (size_t)limb * C::N;
    uint32_t x[R];
    C::load_natural(x, a, tid);
    C::forward(x, sm, tid, q, tw + (size_t)p * C::N);
    C::store_ntt(x, a, tid);
}

template <int LOGN, int R>
__global__ void __launch_bounds__((1 << LOGN) / R) k_ntt_inv(uint32_t *__restrict__ data, PrimeMap pm,
                                                            size_t stride, const PrimeConst *__restrict__ pc,
                                                            const uint2 *__restrict__ tw) {
    using C = NttCore<LOGN, R>;
    extern __shared__ __align__(16) uint32_t sm[];
    const int limb = blockIdx.x, tid = threadIdx.x;
    const int p = prime_of(pm, limb);
    const PrimeConst P = pc[p];
    uint32_t *a = data + blockIdx.y * stride + (size_t)limb * C::N;
    uint32_t x[R];
    C::load_ntt(x, a, tid);
    C::inverse(x, sm, tid, P.q, tw + (size_t)p * C::N, P.ninv, P.ninv_shoup);
    C::store_natural(x, a, tid);
}

// The lazy butterflies' additions selected by each kernel's FMA bits go
// through the FMA pipe (ModQ::one read at run time) in blocks of at most 512
// threads (every block shape in use); in larger blocks the compile-time 1
// folds them back into plain additions (measured slower there).
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
// ModDown's one forward transform a block: every addition on the ALU pipe
// (0.136 against 0.141 ms with the square kernel's choice)
constexpr int kFmaSquare = BCN_FMA_SQ, kFmaKs = BCN_FMA_KS, kFmaMd = 0;

// Pairs of independent transforms run in lockstep (shared twiddle loads and
// barriers, twice the independent work per thread) where the registers allow
// it: 16 residues a thread, at most 512 threads.
template <int LOGN, int R>
constexpr bool kDual = (1 << LOGN) / R <= 512 && R <= 16;

// The key switch's block shape: at N = 8192 (512 threads) two blocks per SM of
// 64 registers and one exchange buffer (digits transformed one at a time)
// measured faster than one block of 128 registers with digit pairs (0.486
// against 0.501 ms per CryptoNets-scale evaluation; the pairs' second buffer
// and the running sums do not fit twice in shared memory); at N = 4096 and
// 16384 the pairs / 128 registers are faster.
template <int LOGN, int R>
constexpr bool kKsWide = LOGN == 13 && R == 16;
template <int LOGN, int R>
constexpr bool kKsDual = kDual<LOGN, R> && !kKsWide<LOGN, R>;
// the one-digit-at-a-time key switch keeps its first running sum in registers
// (the second in shared memory): half the shared-memory traffic of the key
// products (measured 0.483 against 0.486-0.490 ms); at N = 16384 (32 residues a
// thread, 128 registers) it fits as well
#ifndef BCN_KS_REGSUM14
#define BCN_KS_REGSUM14 1  // measured 34.34 against 34.78 ms of key switch per CIFAR-shaped evaluation
#endif
template <int LOGN, int R>
constexpr bool kKsRegSum = kKsWide<LOGN, R> || (BCN_KS_REGSUM14 && LOGN == 14 && R == 32);

// Register budget per thread of the fused kernels (sets their blocks per SM).
#ifndef BCN_CORE_REGS
#define BCN_CORE_REGS 128
#endif
template <int T, int REGS = BCN_CORE_REGS>
struct CoreOcc {
    static constexpr int B = 65536 / (T * REGS);
    static constexpr int MIN_BLOCKS = B > 32 ? 32 : (B < 1 ? 1 : B);
};

// Square activation, first half, one block per (limb, ct): the tensor square
// (c0^2, 2 c0 c1, c1^2) in the NTT domain of the limb's prime.  Y [C][2][n][N]
// is in coefficient form (natural order; transformed here) or, with IN_NTT, in
// the NTT domain (the last-pass layout of the transform).  Out: d0 and d1 in
// the NTT domain (D [C][3][n][N] slots 0 and 1, last-pass layout), d2 in
// coefficient form (slot 2, the key switch's ModUp input: one inverse NTT)
// and, with D2N != nullptr, d2 in the NTT domain too (D2N [C][n][N], which the
// key switch reuses on the digit's own prime).  With `pre` (per limb i, the
// Shoup pair of Dhat_i^{-1} mod q_i of its digit) slot 2 holds d2 Dhat_i^{-1}
// instead.  All outputs canonical.
// grid (n, C).
// Register budget of the square kernel: 64 (two 512-thread blocks per SM at
// N = 8192) measured faster than 128 with either input domain (coefficient
// input: 0.173 against 0.194 ms per CryptoNets-scale evaluation)
// the square kernel's first forward transform (c0), parked in the
// thread-private shared area s1[u T + tid]: a call of its own, so that the
// two transforms' register allocations do not overlap
template <int LOGN, int R>
__device__ __noinline__ void square_park_c0(const uint32_t *__restrict__ y0, uint32_t *sm, uint32_t *s1, int tid,
                                            ModQ mq, const uint2 *__restrict__ tf) {
    using C = NttCore<LOGN, R, true, kFmaSquare>;
    uint32_t x[R];
    C::load_natural(x, y0, tid);
    C::forward(x, sm, tid, mq, tf);
#pragma unroll
    for (int u = 0; u < R; u++) s1[u * C::T + tid] = x[u];
}

template <int T, int REGS>
struct SqnOcc {
    static constexpr int B = 65536 / (T * REGS);
    static constexpr int MIN_BLOCKS = B > 32 ? 32 : (B < 1 ? 1 : B);
};
template <int LOGN, int R, bool IN_NTT>
__global__ void __launch_bounds__((1 << LOGN) / R, IN_NTT ? SqnOcc<(1 << LOGN) / R, 64>::MIN_BLOCKS
                                                          : SqnOcc<(1 << LOGN) / R, R >= 32 ? 128 : 64>::MIN_BLOCKS)
    k_square_core(const uint32_t *__restrict__ Y, uint32_t *__restrict__ D, uint32_t *__restrict__ D2N, int n,
                  const PrimeConst *__restrict__ pc, const uint2 *__restrict__ twf, const uint2 *__restrict__ twi,
                  const uint2 *__restrict__ pre) {
    using C = NttCore<LOGN, R, true, kFmaSquare>;  // data primes only (q < 2^30): lazy butterflies
    constexpr int N = C::N, T = C::T;
    constexpr int V = C::NTT_QUADS ? 4 : (C::NTT_PAIRS ? 2 : 1);  // consecutive NTT-domain elements per register run
    extern __shared__ __align__(16) uint32_t sm[];
    const int i = blockIdx.x, ct = blockIdx.y, tid = threadIdx.x;
    const PrimeConst P = pc[i];
    const uint2 *tf = twf + (size_t)i * N, *ti = twi + (size_t)i * N;
    const ModQ mq(P.q, kFmaOne<LOGN, R> ? P.one : 1u);
    const uint32_t *y0 = Y + (((size_t)ct * 2 + 0) * n + i) * N, *y1 = Y + (((size_t)ct * 2 + 1) * n + i) * N;
    uint32_t *d0 = D + (((size_t)ct * 3 + 0) * n + i) * N, *d1 = D + (((size_t)ct * 3 + 1) * n + i) * N;
    uint32_t *d2 = D + (((size_t)ct * 3 + 2) * n + i) * N;
    uint32_t *d2n = D2N != nullptr ? D2N + ((size_t)ct * n + i) * N : nullptr;
    uint32_t x[R];  // c1^2 / N in the NTT domain, then d2 in coefficient form
    // V consecutive NTT-domain elements (registers u0 .. u0+V-1, any residues
    // below 4q): d0, d1 and d2 stored, c1^2 / N (the inverse NTT's input,
    // whose N^{-1} this folds in) left in x
    auto square_run = [&](const uint32_t(&a)[V], const uint32_t(&b)[V], int u0) {
        uint32_t o0[V], o1[V], o2[V];
#pragma unroll
        for (int z = 0; z < V; z++) {
            const uint32_t aR = shoup_mul(a[z], P.r_mod, P.r_shoup, P.q);
            const uint32_t bR = shoup_mul(b[z], P.r_mod, P.r_shoup, P.q);
            const uint32_t ab = mont_mul(aR, b[z], P.q, P.qneg_inv);
            o0[z] = mont_mul(aR, a[z], P.q, P.qneg_inv);  // c0^2
            o1[z] = add_mod(ab, ab, P.q);                  // 2 c0 c1
            o2[z] = mont_mul(bR, b[z], P.q, P.qneg_inv);  // c1^2
            x[u0 + z] = shoup_mul(o2[z], P.ninv, P.ninv_shoup, P.q);
        }
        const int e = C::ntt_elem(u0, tid);
        if constexpr (V == 4) {
            *reinterpret_cast<uint4 *>(d0 + e) = make_uint4(o0[0], o0[1], o0[2], o0[3]);
            *reinterpret_cast<uint4 *>(d1 + e) = make_uint4(o1[0], o1[1], o1[2], o1[3]);
            if (d2n != nullptr) *reinterpret_cast<uint4 *>(d2n + e) = make_uint4(o2[0], o2[1], o2[2], o2[3]);
        } else if constexpr (V == 2) {
            *reinterpret_cast<uint2 *>(d0 + e) = make_uint2(o0[0], o0[1]);
            *reinterpret_cast<uint2 *>(d1 + e) = make_uint2(o1[0], o1[1]);
            if (d2n != nullptr) *reinterpret_cast<uint2 *>(d2n + e) = make_uint2(o2[0], o2[1]);
        } else {
            d0[e] = o0[0];
            d1[e] = o1[0];
            if (d2n != nullptr) d2n[e] = o2[0];
        }
    };
    if constexpr (IN_NTT) {
#pragma unroll
        for (int u0 = 0; u0 < R; u0 += V) {
            uint32_t a[V], b[V];
            const int e = C::ntt_elem(u0, tid);
            if constexpr (V == 4) {
                *reinterpret_cast<uint4 *>(a) = __ldg(reinterpret_cast<const uint4 *>(y0 + e));
                *reinterpret_cast<uint4 *>(b) = __ldg(reinterpret_cast<const uint4 *>(y1 + e));
            } else if constexpr (V == 2) {
                *reinterpret_cast<uint2 *>(a) = __ldg(reinterpret_cast<const uint2 *>(y0 + e));
                *reinterpret_cast<uint2 *>(b) = __ldg(reinterpret_cast<const uint2 *>(y1 + e));
            } else {
                a[0] = __ldg(y0 + e);
                b[0] = __ldg(y1 + e);
            }
            square_run(a, b, u0);
        }
    } else if constexpr (kDual<LOGN, R>) {
        // c0 and c1 transformed together (two exchange buffers)
        uint32_t y[2][R];
        C::load_natural(y[0], y0, tid);
        C::load_natural(y[1], y1, tid);
        C::forward_n(y, sm, tid, mq, tf);
#pragma unroll
        for (int u0 = 0; u0 < R; u0 += V) {
            uint32_t a[V], b[V];
#pragma unroll
            for (int z = 0; z < V; z++) {
                a[z] = y[0][u0 + z];
                b[z] = y[1][u0 + z];
            }
            square_run(a, b, u0);
        }
    } else {
        // c0 transformed and parked in a thread-private area (u*T + tid), then c1
        uint32_t *s1 = sm + C::SMEM_WORDS;
        square_park_c0<LOGN, R>(y0, sm, s1, tid, mq, tf);
        C::load_natural(x, y1, tid);
        C::forward(x, sm, tid, mq, tf);
#pragma unroll
        for (int u0 = 0; u0 < R; u0 += V) {
            uint32_t a[V], b[V];
#pragma unroll
            for (int z = 0; z < V; z++) {
                a[z] = s1[(u0 + z) * T + tid];
                b[z] = x[u0 + z];
            }
            square_run(a, b, u0);
        }
    }
    C::inverse_unscaled(x, sm, tid, mq, ti);
    if (pre != nullptr) {  // d2 Dhat_i^{-1} mod q_i, the key switch's ModUp factor of this limb
        const uint2 f = pre[i];
#pragma unroll
        for (int u = 0; u < R; u++) x[u] = shoup_mul(x[u], f.x, f.y, P.q);
    }
    C::store_natural(x, d2, tid);
}

// ModUp residue of digit j (primes q_lo .. q_{hi-1}, lo = j alpha) of the
// polynomial x2 ([n][N] coefficient form, canonical) in target prime t (prime
// index pt, constants P), in the pass-0 distribution of NttCore<LOGN, R>, ready
// for the forward NTT: on the digit's own primes the residue itself; else the
// centred fast basis conversion
//     sum_u r_u * Dhat_u - #{u : r_u > (q_u-1)/2} * D_j,  r_u = [x_u Dhat_u^{-1}]_{q_u},
// which for one-prime digits is d mod t, less q_j mod t when d > (q_j-1)/2.
// With LAZY (t a data prime) one-prime digits leave d + (t - q_j mod t) < 3t
// and digits of two primes a residue below 4t, valid lazy NTT inputs;
// otherwise the residue is canonical.  With PRE the
// limbs of multi-prime digits already hold r_u = [x_u Dhat_u^{-1}]_{q_u} (the
// square kernel's output for the key switch: computed there once instead of
// once per target prime); the digit's own primes are then never read here.
template <int LOGN, int R, bool LAZY, bool PRE = false>
__device__ __forceinline__ void modup_residue(uint32_t (&x)[R], const uint32_t *__restrict__ x2, int t, int pt,
                                              int j, int n, const KsDev &ks, const PrimeConst *__restrict__ pc,
                                              const PrimeConst &P, int tid) {
    using C = NttCore<LOGN, R>;
    constexpr int N = C::N;
    const int A = ks.alpha, lo = j * A, hi = min(lo + A, n);
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
    } else if (LAZY && hi - lo <= 2) {
        // digits of two primes (and a last digit of one) on a data prime, lazily:
        // the Shoup products' sum (below 4t) folded once into [0, 2t), then
        // t - (D_j mod t) added once per centred correction, which keeps the
        // residue below 4t, a valid lazy NTT input congruent to the canonical one
        const size_t jb = (size_t)(n * ks.dnum_max + j);
        const uint32_t tmq = P.q - ks.dprod[jb * ks.P + pt], q2 = 2 * P.q;
        const uint32_t q0 = pc[lo].q, half0 = pc[lo].half;
        const uint2 di0 = ks.dhat_inv[jb * A], dh0 = ks.dhat[(jb * A) * ks.P + pt];
        const uint32_t *x0 = x2 + (size_t)lo * N;
        if (hi - lo == 2) {
            const uint32_t q1 = pc[lo + 1].q, half1 = pc[lo + 1].half;
            const uint2 di1 = ks.dhat_inv[jb * A + 1], dh1 = ks.dhat[(jb * A + 1) * ks.P + pt];
            const uint32_t *x1 = x0 + N;
#pragma unroll
            for (int u = 0; u < R; u++) {
                const int e = C::nat_elem(u, tid);
                const uint32_t a0 = __ldg(x0 + e), a1 = __ldg(x1 + e);
                const uint32_t r0 = PRE ? a0 : shoup_mul(a0, di0.x, di0.y, q0);
                const uint32_t r1 = PRE ? a1 : shoup_mul(a1, di1.x, di1.y, q1);
                uint32_t y = shoup_mul_lazy(r0, dh0.x, dh0.y, P.q) + shoup_mul_lazy(r1, dh1.x, dh1.y, P.q);
                y = min(y, y - q2);
                y += r0 > half0 ? tmq : 0u;
                y += r1 > half1 ? tmq : 0u;
                x[u] = y;
            }
        } else {
#pragma unroll
            for (int u = 0; u < R; u++) {
                const uint32_t a0 = __ldg(x0 + C::nat_elem(u, tid));
                const uint32_t r0 = PRE ? a0 : shoup_mul(a0, di0.x, di0.y, q0);
                x[u] = shoup_mul_lazy(r0, dh0.x, dh0.y, P.q) + (r0 > half0 ? tmq : 0u);  // < 3t
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
                const uint32_t raw = __ldg(xi + C::nat_elem(u, tid));
                const uint32_t r = PRE ? raw : shoup_mul(raw, di.x, di.y, qi);
                uint32_t y = add_mod(x[u], shoup_mul(r, dh.x, dh.y, P.q), P.q);
                if (r > half) y = sub_mod(y, dp, P.q);
                x[u] = y;
            }
        }
    }
}

// Key switching of d2, fused per (target prime t, ciphertext): for every
// digit j, ModUp of d2 into prime t (the residue itself on the digit's own
// primes -- taken from D2N in the NTT domain when given -- else the centred
// fast basis conversion
//     sum_u r_u * Dhat_u - #{u : r_u > (q_u-1)/2} * D_j,  r_u = [x_u Dhat_u^{-1}]_{q_u},
// which for one-prime digits is d mod t, less q_j mod t when d > (q_j-1)/2),
// forward NTT, and the product with evk_j (prepared as k*R*N^{-1}, so one
// Montgomery product gives k*x/N) accumulated for both key halves; then the
// inverse NTT of the two sums -- or, with ntt_out, on the data primes below
// the top one the sums times N left in the NTT domain (last-pass layout), and
// on the top prime the rescale's INTT(A_top P^{-1} + D_top).  No extended-basis
// limb is stored.  D [C][3][n][N] (d2 in coefficient form; with ntt_out, d0
// and d1 in the NTT domain) -> ACC [C][2][n+K][N] (coefficient form; with
// ntt_out the first n-1 limbs of each poly in the NTT domain).
template <int LOGN, int R, bool LAZY>
__device__ __forceinline__ void ks_core_body(const uint32_t *__restrict__ D, const uint32_t *__restrict__ D2N,
                                             const uint32_t *__restrict__ evk, uint32_t *__restrict__ acc_out,
                                             int n, int ntt_out, int pre, const KsDev &ks,
                                             const PrimeConst *__restrict__ pc, const uint2 *__restrict__ twf,
                                             const uint2 *__restrict__ twi) {
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
    uint32_t *s0 = sm + (kKsDual<LOGN, R> ? 2 : 1) * C::SMEM_WORDS, *s1 = s0 + N;
    const int t = blockIdx.x, ct = blockIdx.y, tid = threadIdx.x;
    uint32_t r0[kKsRegSum<LOGN, R> ? R : 1];  // the first sum, when it lives in registers
    auto S0 = [&](int u) -> uint32_t & {
        if constexpr (kKsRegSum<LOGN, R>)
            return r0[u];
        else
            return s0[u * T + tid];
    };
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
                for (int z = 0; z < 4; z++) ks_accumulate(S0(u + z), s1[(u + z) * T + tid], xr[u + z],
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
                for (int z = 0; z < 2; z++) ks_accumulate(S0(u + z), s1[(u + z) * T + tid], xr[u + z],
                                                          w0[z], w1[z], P);
            }
        } else {
#pragma unroll
            for (int u = 0; u < R; u++) {
                const int e = C::ntt_elem(u, tid);
                ks_accumulate(S0(u), s1[u * T + tid], xr[u], __ldg(k0 + e), __ldg(k1 + e), P);
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
                uint32_t a0 = S0(u + z), a1 = s1[(u + z) * T + tid];
                ks_accumulate(a0, a1, xr[0][u + z], wa0[z], wa1[z], P);
                ks_accumulate(a0, a1, xr[1][u + z], wb0[z], wb1[z], P);
                S0(u + z) = a0;
                s1[(u + z) * T + tid] = a1;
            }
        }
    };
    uint32_t x[R];
#pragma unroll
    for (int u = 0; u < R; u++) S0(u) = s1[u * T + tid] = 0;
    bool summed = false;
    if constexpr (LAZY && kKsDual<LOGN, R>) {
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
            if (pre)
                modup_residue<LOGN, R, LAZY, true>(x, x2, t, pt, j, n, ks, pc, P, tid);
            else
                modup_residue<LOGN, R, LAZY>(x, x2, t, pt, j, n, ks, pc, P, tid);
            C::forward(x, sm, tid, ModQ(P.q, kFmaOne<LOGN, R> ? P.one : 1u), tf);
        }
        key_product(x, j);
    }
    // with ntt_out, the data primes' sums below the top prime stay in the NTT
    // domain: times N (the key carries N^{-1} for the inverse transform),
    // canonical, last-pass layout.  On the top prime q_{n-1} the block folds in
    // the rescale's first step: INTT(A_top P^{-1} + D_top) in coefficient form,
    // i.e. the unscaled inverse of s P^{-1} + D_top N^{-1} (D_top: d0 or d1 of
    // the square, NTT domain), stored in place of the sums.
    const bool to_ntt = ntt_out && t < n - 1, top_fold = ntt_out && t == n - 1;
    // s P^{-1} + D_top N^{-1} for poly b, registers u .. u+V-1 (NTT domain)
    auto fold = [&](uint32_t(&y)[R], int b) {
        const uint2 pi = ks.pinv[t];
        const uint32_t *dt = D + (((size_t)ct * 3 + b) * n + t) * N;
        constexpr int V = C::NTT_QUADS ? 4 : (C::NTT_PAIRS ? 2 : 1);
#pragma unroll
        for (int u0 = 0; u0 < R; u0 += V) {
            uint32_t dv[V];
            const int e = C::ntt_elem(u0, tid);
            if constexpr (V == 4)
                *reinterpret_cast<uint4 *>(dv) = __ldg(reinterpret_cast<const uint4 *>(dt + e));
            else if constexpr (V == 2)
                *reinterpret_cast<uint2 *>(dv) = __ldg(reinterpret_cast<const uint2 *>(dt + e));
            else
                dv[0] = __ldg(dt + e);
#pragma unroll
            for (int z = 0; z < V; z++)
                y[u0 + z] = add_mod(shoup_mul(y[u0 + z], pi.x, pi.y, P.q),
                                    shoup_mul(dv[z], P.ninv, P.ninv_shoup, P.q), P.q);
        }
    };
    if constexpr (kKsDual<LOGN, R>) {
        uint32_t y[2][R];
#pragma unroll
        for (int u = 0; u < R; u++) {
            y[0][u] = S0(u);
            y[1][u] = s1[u * T + tid];
        }
        if (top_fold) {
            fold(y[0], 0);
            fold(y[1], 1);
        }
        if (to_ntt) {
#pragma unroll
            for (int u = 0; u < R; u++) {
                y[0][u] = shoup_mul(y[0][u], P.nmod, P.nmod_shoup, P.q);
                y[1][u] = shoup_mul(y[1][u], P.nmod, P.nmod_shoup, P.q);
            }
            C::store_ntt(y[0], acc_out + (((size_t)ct * 2 + 0) * nb + t) * N, tid);
            C::store_ntt(y[1], acc_out + (((size_t)ct * 2 + 1) * nb + t) * N, tid);
            return;
        }
        C::inverse_unscaled_n(y, sm, tid, ModQ(P.q, kFmaOne<LOGN, R> ? P.one : 1u), ti);
        C::store_natural(y[0], acc_out + (((size_t)ct * 2 + 0) * nb + t) * N, tid);
        C::store_natural(y[1], acc_out + (((size_t)ct * 2 + 1) * nb + t) * N, tid);
        return;
    }
#pragma unroll
    for (int b = 0; b < 2; b++) {
        uint32_t *dst = acc_out + (((size_t)ct * 2 + b) * nb + t) * N;
#pragma unroll
        for (int u = 0; u < R; u++) x[u] = b == 0 ? S0(u) : s1[u * T + tid];
        if (top_fold) fold(x, b);
        if (to_ntt) {
#pragma unroll
            for (int u = 0; u < R; u++) x[u] = shoup_mul(x[u], P.nmod, P.nmod_shoup, P.q);
            C::store_ntt(x, dst, tid);
        } else {
            C::inverse_unscaled(x, sm, tid, ModQ(P.q, kFmaOne<LOGN, R> ? P.one : 1u), ti);
            C::store_natural(x, dst, tid);
        }
    }
}

// grid (n+K, C); lazy butterflies for the data primes (< 2^30), strict ones for
// the special primes (< 2^31)
template <int LOGN, int R>
__global__ void __launch_bounds__((1 << LOGN) / R, CoreOcc<(1 << LOGN) / R, kKsWide<LOGN, R> ? 64 : BCN_CORE_REGS>::MIN_BLOCKS)
    k_ks_core(const uint32_t *__restrict__ D, const uint32_t *__restrict__ D2N, const uint32_t *__restrict__ evk,
              uint32_t *__restrict__ acc_out, int n, int ntt_out, int pre, KsDev ks,
              const PrimeConst *__restrict__ pc, const uint2 *__restrict__ twf, const uint2 *__restrict__ twi) {
    const int t = blockIdx.x;
    const int pt = t < n ? t : ks.L + (t - n);
    if (pc[pt].q < (1u << 30))
        ks_core_body<LOGN, R, true>(D, D2N, evk, acc_out, n, ntt_out, pre, ks, pc, twf, twi);
    else
        ks_core_body<LOGN, R, false>(D, D2N, evk, acc_out, n, ntt_out, pre, ks, pc, twf, twi);
}

// ModDown by P and rescale by the top prime q_top = q_{n-1} in the NTT domain
// (App. A of the paper: relinearisation ends with the division by P, the
// square activation with the rescale; the two roundings in sequence, as the
// coefficient-form definition states them):
//   c_i   = (a_i - conv_i(a_P)) P^{-1} + d_i        ModDown, every limb i < n
//   out_i = (c_i - [c_top]) q_top^{-1}                rescale, i < n - 1
// where conv_i(a_P) = sum_m r_m Phat_m - #{m : r_m > (p_m - 1)/2} P (mod q_i),
// r_m = [a_{P,m} Phat_m^{-1}]_{p_m}, is the centred fast basis conversion of the
// special-prime limbs (coefficient form) and [c_top] the centred lift of the
// top limb.  The NTT is linear, so with A_i, D_i the NTT-domain a_i, d_i:
//   c_top = INTT(A_top P^{-1} + D_top) - conv_top(a_P) P^{-1}
//   out_i = (A_i P^{-1} + D_i - NTT(conv_i(a_P) P^{-1} + [c_top])) q_top^{-1}
// The inverse NTT of c_top is the key switch's (its block on the top prime
// forms INTT(A_top P^{-1} + D_top)); what is left is one forward NTT per limb
// and poly.  The results equal the NTT of the coefficient-form ModDown and
// rescale, residue for residue.

// out_i of polys b0 .. b0+NP-1 of ciphertext ct, i < n - 1 (NP = 2: both
// polys transformed in lockstep).  D [C][3][n][N] (slots 0, 1: d0, d1 in the
// NTT domain), ACC [C][2][n+K][N] (limbs i < n-1: A_i in the NTT domain; limb
// n-1: c_top = INTT(A_top P^{-1} + D_top) - conv_top(a_P) P^{-1}, coefficient
// form, from the key switch and k_md_top;
// limbs n..n+K-1: a_P times Phat_m^{-1} -- the key carries that factor --,
// coefficient form) -> OUT [C][2][n-1][N] (NTT domain,
// last-pass layout, canonical).  grid (n - 1, 2 / NP, C)
// Register budget of the ModDown/rescale blocks: its element-wise prologue
// (loads of the special-prime limbs and the top limb) wants occupancy --
// measured at N = 8192: 40 registers (3 blocks per SM) 0.140 ms, 64 registers
// 0.155 ms, 128 registers 0.193 ms; 32 residues a thread need 64
// The top limb's part of ModDown and rescale, the same for every limb i:
// c_top = acc_top - conv_top(a_P) P^{-1} (mod q_top), stored over acc_top
// (limb n-1 of ACC) for k_md_limb to lift; once per (coefficient, poly,
// ciphertext) instead of once per limb.  Four coefficients a thread.
// grid (N/4/256, 2, C)
template <int K>
__global__ void __launch_bounds__(256) k_md_top(uint32_t *__restrict__ acc, int n, int N, KsDev ks,
                                                const PrimeConst *__restrict__ pc) {
    const int k4 = blockIdx.x * blockDim.x + threadIdx.x;
    if (k4 * 4 >= N) return;
    const int b = blockIdx.y, ct = blockIdx.z, nb = n + K, top = n - 1;
    const uint32_t qtop = pc[top].q, pmod_t = ks.pmod[top];
    const uint2 pit = ks.pinv[top];
    uint32_t *row = acc + ((size_t)ct * 2 + b) * nb * N;
    uint32_t conv[4] = {0, 0, 0, 0};
    int cnt[4] = {0, 0, 0, 0};
#pragma unroll
    for (int m = 0; m < K; m++) {
        const uint32_t ph2 = pc[ks.L + m].half;
        const uint2 pht = ks.phat[(size_t)m * ks.L + top];
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(row + (size_t)(n + m) * N) + k4);  // a_m Phat_m^{-1}
        const uint32_t r[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int z = 0; z < 4; z++) {
            cnt[z] += r[z] > ph2;
            conv[z] = add_mod(conv[z], shoup_mul(r[z], pht.x, pht.y, qtop), qtop);
        }
    }
    uint4 *tp = reinterpret_cast<uint4 *>(row + (size_t)top * N) + k4;
    const uint4 a = *tp;
    const uint32_t av[4] = {a.x, a.y, a.z, a.w};
    uint32_t y[4];
#pragma unroll
    for (int z = 0; z < 4; z++) {
#pragma unroll
        for (int c = 0; c < K; c++) conv[z] = c < cnt[z] ? sub_mod(conv[z], pmod_t, qtop) : conv[z];
        y[z] = sub_mod(av[z], shoup_mul(conv[z], pit.x, pit.y, qtop), qtop);
    }
    *tp = make_uint4(y[0], y[1], y[2], y[3]);
}

template <int T, int R>
struct MdOcc {
    static constexpr int REGS = R >= 32 ? 64 : 40;
    static constexpr int B = 65536 / (T * REGS);
    static constexpr int MIN_BLOCKS = B > 32 ? 32 : (B < 1 ? 1 : B);
};
template <int LOGN, int R, int NP, int K>
__global__ void __launch_bounds__((1 << LOGN) / R, NP == 1 ? MdOcc<(1 << LOGN) / R, R>::MIN_BLOCKS
                                                           : CoreOcc<(1 << LOGN) / R>::MIN_BLOCKS)
    k_md_limb(const uint32_t *__restrict__ D, const uint32_t *__restrict__ acc, uint32_t *__restrict__ out, int n,
              KsDev ks, const PrimeConst *__restrict__ pc, const uint2 *__restrict__ twf) {
    using C = NttCore<LOGN, R, true, kFmaMd>;  // data primes: lazy butterflies
    constexpr int N = C::N;
    constexpr int V = C::NTT_QUADS ? 4 : (C::NTT_PAIRS ? 2 : 1);
    extern __shared__ __align__(16) uint32_t sm[];
    const int i = blockIdx.x, b0 = blockIdx.y * NP, ct = blockIdx.z, tid = threadIdx.x;
    const int nb = n + ks.K, top = n - 1;
    const PrimeConst P = pc[i];
    const uint32_t qtop = pc[top].q, htop = pc[top].half, tmq = P.q - qtop;  // q_i > q_top
    const uint2 pi = ks.pinv[i], qti = ks.qtop_inv[(size_t)top * ks.L + i];
    const uint32_t pmod_i = ks.pmod[i];
    const uint32_t *row[NP];
#pragma unroll
    for (int p = 0; p < NP; p++) row[p] = acc + ((size_t)ct * 2 + b0 + p) * nb * N;
    // the epilogue's rows A_i and D_i, requested into L2 now: the prologue and
    // the transform run meanwhile (measured at N = 16384: ModDown 9.50 to 9.20
    // ms per CIFAR-shaped evaluation; no gain at N = 8192)
    if constexpr (N >= 16384) {
#pragma unroll
        for (int p = 0; p < NP; p++) {
            prefetch_row_l2(row[p] + (size_t)i * N, N, tid, C::T);
            prefetch_row_l2(D + (((size_t)ct * 3 + b0 + p) * n + i) * N, N, tid, C::T);
        }
    }
    // coefficient form: conv_i(a_P) P^{-1} + [c_top] (mod q_i), with
    // c_top = acc_top - conv_top(a_P) P^{-1} (mod q_top) formed by k_md_top
    uint32_t x[NP][R];
#pragma unroll
    for (int u = 0; u < R; u++) {
        const int e = C::nat_elem(u, tid);
#pragma unroll
        for (int p = 0; p < NP; p++) {
            // K (the number of special primes) is a template parameter and the
            // correction below a chain of selects: no branch, so the loads of
            // all R elements can be issued together
            uint32_t conv_i = 0;
            if constexpr (K <= 2) {
                // lazily: the Shoup products' sum folded once into [0, 2q), plus
                // q - (P mod q_i) per centred correction (below 4q), times P^{-1}
                // up to one q, plus the lift: below 3q, a valid lazy NTT input
                // congruent to the canonical value
                uint32_t corr = 0;
#pragma unroll
                for (int m = 0; m < K; m++) {
                    const uint2 phi = ks.phat[(size_t)m * ks.L + i];
                    // a_m Phat_m^{-1}: the prepared key's special-prime limbs carry Phat_m^{-1}
                    const uint32_t r = __ldg(row[p] + (size_t)(n + m) * N + e);
                    conv_i += shoup_mul_lazy(r, phi.x, phi.y, P.q);
                    if (m > 0) conv_i = min(conv_i, conv_i - 2 * P.q);
                    corr += r > pc[ks.L + m].half ? P.q - pmod_i : 0u;
                }
                const uint32_t y = __ldg(row[p] + (size_t)top * N + e);  // c_top (k_md_top)
                x[p][u] = shoup_mul_lazy(conv_i + corr, pi.x, pi.y, P.q) + (y > htop ? y + tmq : y);
            } else {
                int cnt = 0;
#pragma unroll
                for (int m = 0; m < K; m++) {
                    const uint32_t ph2 = pc[ks.L + m].half;
                    const uint2 phi = ks.phat[(size_t)m * ks.L + i];
                    const uint32_t r = __ldg(row[p] + (size_t)(n + m) * N + e);
                    cnt += r > ph2;
                    conv_i = add_mod(conv_i, shoup_mul(r, phi.x, phi.y, P.q), P.q);
                }
#pragma unroll
                for (int c = 0; c < K; c++) conv_i = c < cnt ? sub_mod(conv_i, pmod_i, P.q) : conv_i;
                const uint32_t y = __ldg(row[p] + (size_t)top * N + e);  // c_top (k_md_top)
                const uint32_t lift = y > htop ? y + tmq : y;
                x[p][u] = add_mod(shoup_mul(conv_i, pi.x, pi.y, P.q), lift, P.q);
            }
        }
    }
    C::template forward_n<NP>(x, sm, tid, ModQ(P.q, kFmaOne<LOGN, R> ? P.one : 1u), twf + (size_t)i * N);  // [0, 4q)
    const uint32_t q2 = 2 * P.q;
#pragma unroll
    for (int p = 0; p < NP; p++) {
        const uint32_t *A = row[p] + (size_t)i * N;
        const uint32_t *Di = D + (((size_t)ct * 3 + b0 + p) * n + i) * N;
        uint32_t *o = out + (((size_t)ct * 2 + b0 + p) * (n - 1) + i) * N;
#pragma unroll
        for (int u0 = 0; u0 < R; u0 += V) {
            const int e = C::ntt_elem(u0, tid);
            uint32_t av[V], dv[V], r[V];
            if constexpr (V == 4) {
                *reinterpret_cast<uint4 *>(av) = __ldg(reinterpret_cast<const uint4 *>(A + e));
                *reinterpret_cast<uint4 *>(dv) = __ldg(reinterpret_cast<const uint4 *>(Di + e));
            } else if constexpr (V == 2) {
                *reinterpret_cast<uint2 *>(av) = __ldg(reinterpret_cast<const uint2 *>(A + e));
                *reinterpret_cast<uint2 *>(dv) = __ldg(reinterpret_cast<const uint2 *>(Di + e));
            } else {
                av[0] = __ldg(A + e);
                dv[0] = __ldg(Di + e);
            }
#pragma unroll
            for (int z = 0; z < V; z++) {
                uint32_t f = x[p][u0 + z] >= q2 ? x[p][u0 + z] - q2 : x[p][u0 + z];
                f = f >= P.q ? f - P.q : f;
                const uint32_t c = add_mod(shoup_mul(av[z], pi.x, pi.y, P.q), dv[z], P.q);
                r[z] = shoup_mul(sub_mod(c, f, P.q), qti.x, qti.y, P.q);
            }
            if constexpr (V == 4)
                *reinterpret_cast<uint4 *>(o + e) = make_uint4(r[0], r[1], r[2], r[3]);
            else if constexpr (V == 2)
                *reinterpret_cast<uint2 *>(o + e) = make_uint2(r[0], r[1]);
            else
                o[e] = r[0];
        }
    }
}

// ------------------------------------------------------------ hoisted rotations
// Rotations of one ciphertext by many steps share their ModUp (App. D builds
// packed convolutions and dense layers from many rotations of the same
// ciphertext).  The automorphism sigma_g acts on a limb's coefficients as a
// signed permutation, the centred lift is odd (q odd) and the fast basis
// conversion linear, so ModUp(sigma_g(c1)) = sigma_g(ModUp(c1)) residue for
// residue: one ModUp of c1, kept in the NTT domain, serves every rotation, and
// in the NTT domain sigma_g is a plain permutation of the evaluation points.
// The results equal those of rotating one step at a time, bit for bit.

// U [C][dnum][n+K][N] <- ModUp of digit j of the ciphertexts' c1 (in
// [C][2][n][N], coefficient form) into target prime t, forward NTT (last-pass
// layout; lazy values below 4q on the data primes, canonical on the special
// primes).  grid (n+K, dnum, C)
template <int LOGN, int R, bool LAZY>
__device__ __forceinline__ void modup_hoist_body(const uint32_t *__restrict__ in, uint32_t *__restrict__ U, int n,
                                                 const KsDev &ks, const PrimeConst *__restrict__ pc,
                                                 const uint2 *__restrict__ twf) {
    using C = NttCore<LOGN, R, LAZY, kFmaKs>;
    constexpr int N = C::N;
    extern __shared__ __align__(16) uint32_t sm[];
    const int t = blockIdx.x, j = blockIdx.y, ct = blockIdx.z, tid = threadIdx.x;
    const int nb = n + ks.K, dnum = (n + ks.alpha - 1) / ks.alpha;
    const int pt = t < n ? t : ks.L + (t - n);
    const PrimeConst P = pc[pt];
    const uint32_t *x2 = in + ((size_t)ct * 2 + 1) * n * N;
    uint32_t x[R];
    modup_residue<LOGN, R, LAZY>(x, x2, t, pt, j, n, ks, pc, P, tid);
    C::forward(x, sm, tid, ModQ(P.q, kFmaOne<LOGN, R> ? P.one : 1u), twf + (size_t)pt * N);
    C::store_ntt(x, U + (((size_t)ct * dnum + j) * nb + t) * N, tid);
}

template <int LOGN, int R>
__global__ void __launch_bounds__((1 << LOGN) / R) k_modup_hoist(const uint32_t *__restrict__ in,
                                                                 uint32_t *__restrict__ U, int n, KsDev ks,
                                                                 const PrimeConst *__restrict__ pc,
                                                                 const uint2 *__restrict__ twf) {
    const int t = blockIdx.x;
    const int pt = t < n ? t : ks.L + (t - n);
    if (pc[pt].q < (1u << 30))
        modup_hoist_body<LOGN, R, true>(in, U, n, ks, pc, twf);
    else
        modup_hoist_body<LOGN, R, false>(in, U, n, ks, pc, twf);
}

// NTT-domain element whose value sigma_g moves to element e: with the
// evaluation point psi^(2 brv(e) + 1) at element e, sigma_g(a) there is a at
// psi^((2 brv(e) + 1) g) = psi^(2 k + 1), held by element brv(k).
template <int LOGN>
__device__ __forceinline__ int auto_ntt_src(int e, uint32_t g) {
    const uint32_t k = __brev((uint32_t)e) >> (32 - LOGN);
    const uint32_t m = ((2 * k + 1) * g) & ((2u << LOGN) - 1);
    return (int)(__brev((m - 1) >> 1) >> (32 - LOGN));
}

// Key switching of sigma_g(c1) for a batch of rotations, from the hoisted U:
// for every digit j the limb U[ct][j][t] is staged in shared memory, gathered
// through the permutation of sigma_g, multiplied by both halves of the
// rotation's Galois key (prepared form: k R N^{-1}, NTT domain) and added to
// two running sums, whose inverse NTT (the key's N^{-1} folded in) gives
// ACC [C][count][2][n+K][N] in coefficient form, as the key-switching core
// leaves it for ModDown.  grid (n+K, count, C)
template <int LOGN, int R, bool LAZY>
__device__ __forceinline__ void ks_rot_body(const uint32_t *__restrict__ U, RotBatch rb,
                                            uint32_t *__restrict__ acc_out, int n, const KsDev &ks,
                                            const PrimeConst *__restrict__ pc, const uint2 *__restrict__ twi) {
    using C = NttCore<LOGN, R, LAZY, kFmaKs>;
    constexpr int N = C::N, T = C::T;
    extern __shared__ __align__(16) uint32_t sm[];
    uint32_t *s0 = sm + C::SMEM_WORDS, *s1 = s0 + N;  // running sums, thread-private slots u*T + tid
    const int t = blockIdx.x, r = blockIdx.y, ct = blockIdx.z, tid = threadIdx.x;
    const int nb = n + ks.K, dnum = (n + ks.alpha - 1) / ks.alpha;
    const int pt = t < n ? t : ks.L + (t - n);
    const PrimeConst P = pc[pt];
    const uint32_t g = rb.g[r];
    const uint32_t *key = rb.gk[r];
#pragma unroll
    for (int u = 0; u < R; u++) s0[u * T + tid] = s1[u * T + tid] = 0;
    for (int j = 0; j < dnum; j++) {
        const uint32_t *src = U + (((size_t)ct * dnum + j) * nb + t) * N;
        __syncthreads();  // the previous digit's gathers are done
        for (int e = 4 * tid; e < N; e += 4 * T) {
            const uint4 v = __ldg(reinterpret_cast<const uint4 *>(src + e));
            const int pe = C::padded(e);  // e..e+3 lie in one run of 32
            sm[pe] = v.x;
            sm[pe + 1] = v.y;
            sm[pe + 2] = v.z;
            sm[pe + 3] = v.w;
        }
        __syncthreads();
        const uint32_t *k0 = key + ((size_t)(j * 2 + 0) * ks.P + pt) * N;
        const uint32_t *k1 = key + ((size_t)(j * 2 + 1) * ks.P + pt) * N;
        // one element at a time: gathered through sigma_g, multiplied, added
#pragma unroll 4
        for (int u = 0; u < R; u++) {
            const int e = C::ntt_elem(u, tid);
            const uint32_t xv = sm[C::padded(auto_ntt_src<LOGN>(e, g))];
            const uint32_t w0 = __ldg(k0 + e), w1 = __ldg(k1 + e);
            uint32_t &a0 = s0[u * T + tid], &a1 = s1[u * T + tid];
            if constexpr (LAZY) {  // sums in [0, 2q) (the lazy inverse NTT's input range)
                const uint32_t nq2 = 0u - 2 * P.q;
                const uint32_t v0 = mont_mul_lazy(xv, w0, P.q, P.qneg_inv) + a0;
                const uint32_t v1 = mont_mul_lazy(xv, w1, P.q, P.qneg_inv) + a1;
                a0 = min(v0, v0 + nq2);
                a1 = min(v1, v1 + nq2);
            } else {
                a0 = add_mod(a0, mont_mul(xv, w0, P.q, P.qneg_inv), P.q);
                a1 = add_mod(a1, mont_mul(xv, w1, P.q, P.qneg_inv), P.q);
            }
        }
    }
    // the gathers read the staged limb at any position; the inverse NTT's first
    // exchange is warp-local and writes without a block barrier of its own
    __syncthreads();
    uint32_t x[R];
#pragma unroll 1
    for (int b = 0; b < 2; b++) {
        const uint32_t *sb = b == 0 ? s0 : s1;
#pragma unroll
        for (int u = 0; u < R; u++) x[u] = sb[u * T + tid];
        C::inverse_unscaled(x, sm, tid, ModQ(P.q, kFmaOne<LOGN, R> ? P.one : 1u), twi + (size_t)pt * N);
        C::store_natural(x, acc_out + ((((size_t)ct * rb.count + r) * 2 + b) * nb + t) * N, tid);
    }
}

template <int LOGN, int R>
__global__ void __launch_bounds__((1 << LOGN) / R) k_ks_rot(const uint32_t *__restrict__ U, RotBatch rb,
                                                            uint32_t *__restrict__ acc_out, int n, KsDev ks,
                                                            const PrimeConst *__restrict__ pc,
                                                            const uint2 *__restrict__ twi) {
    const int t = blockIdx.x;
    const int pt = t < n ? t : ks.L + (t - n);
    if (pc[pt].q < (1u << 30))
        ks_rot_body<LOGN, R, true>(U, rb, acc_out, n, ks, pc, twi);
    else
        ks_rot_body<LOGN, R, false>(U, rb, acc_out, n, ks, pc, twi);
}

// R residues per thread for the NTT and square kernels, RKS for the key switch
template <int LOGN, int R, int RKS = R>
struct CoreImpl {
    using Core = NttCore<LOGN, R>;
    using CoreKs = NttCore<LOGN, RKS>;
    static constexpr size_t SMEM = (size_t)Core::SMEM_WORDS * 4;            // NTT alone
    // NTT alone; + two parking areas (or a second exchange buffer and one)
    // square kernel, coefficient input: two exchange buffers, or one and a parking area
    static constexpr size_t SMEM3 = ((size_t)(kDual<LOGN, R> ? 2 : 1) * Core::SMEM_WORDS + (kDual<LOGN, R> ? 0 : Core::N)) * 4;
    // square kernel, NTT-domain input: the inverse transform of d2 alone
    static constexpr size_t SMEM_SQ_NTT = SMEM;
    // ModDown/rescale: the square kernel's block shape up to N = 8192, else
    // the key switch's
    // (one poly per block measured faster than two in lockstep: the kernel's
    // element-wise prologue wants the occupancy of 64-register blocks)
    static constexpr int RMD = kDual<LOGN, R> ? R : RKS;
    static constexpr int MD_NP = 1;
    using CoreMd = NttCore<LOGN, RMD>;
    static constexpr size_t SMEM_MD = (size_t)MD_NP * CoreMd::SMEM_WORDS * 4;
    // key switch: exchange buffer(s) and the two running sums
    static constexpr size_t SMEM_KS = ((size_t)(kKsDual<LOGN, RKS> ? 2 : 1) * CoreKs::SMEM_WORDS + 2 * CoreKs::N) * 4;
    // hoisted rotations (key switch's block shape): ModUp, one exchange buffer;
    // rotation key products, the staging / exchange buffer and the two sums
    static constexpr size_t SMEM_HOIST = (size_t)CoreKs::SMEM_WORDS * 4;
    static constexpr size_t SMEM_KSROT = ((size_t)CoreKs::SMEM_WORDS + 2 * CoreKs::N) * 4;

    static bcn_status ntt(const bcn_ctx *c, uint32_t *data, size_t n_limbs, size_t n_groups, size_t stride,
                          PrimeMap pm, bool inverse, cudaStream_t st) {
        if (n_limbs == 0 || n_groups == 0) return BCN_OK;
        if (n_limbs > 0x7FFFFFFFull || n_groups > 65535) return fail(BCN_E_INVAL, "NTT launch too large");
        const dim3 grid((unsigned)n_limbs, (unsigned)n_groups);
        if (inverse)
            k_ntt_inv<LOGN, R><<<grid, Core::T, SMEM, st>>>(data, pm, stride, c->d_pc, c->d_tw_inv);
        else
            k_ntt_fwd<LOGN, R><<<grid, Core::T, SMEM, st>>>(data, pm, stride, c->d_pc, c->d_tw_fwd);
        return check_launch("NTT");
    }
    // Digits of more than one prime, with the NTT-domain d2 kept for the key
    // switch's own primes: the square kernel stores d2 times each limb's ModUp
    // factor Dhat_i^{-1} and the key switch reads it as is (both sides decide
    // alike from alpha and D2N)
    static const uint2 *modup_pre(const bcn_ctx *c, int n, const uint32_t *D2N) {
        if (c->alpha < 2 || D2N == nullptr) return nullptr;
        const KsDev ks = ks_dev(c);
        return ks.dhat_inv + (size_t)n * ks.dnum_max * ks.alpha;  // [(n dnum_max + j) alpha + v] at limb j alpha + v
    }
    static bcn_status square(const bcn_ctx *c, int n, const uint32_t *Y, uint32_t *D, uint32_t *D2N, int C,
                             bool in_ntt, cudaStream_t st) {
        const uint2 *pre = modup_pre(c, n, D2N);
        if (in_ntt)
            k_square_core<LOGN, R, true><<<dim3(n, C), Core::T, SMEM_SQ_NTT, st>>>(Y, D, D2N, n, c->d_pc, c->d_tw_fwd,
                                                                                c->d_tw_inv, pre);
        else
            k_square_core<LOGN, R, false><<<dim3(n, C), Core::T, SMEM3, st>>>(Y, D, D2N, n, c->d_pc, c->d_tw_fwd,
                                                                           c->d_tw_inv, pre);
        return check_launch("k_square_core");
    }
    static bcn_status keyswitch(const bcn_ctx *c, int n, const uint32_t *D, const uint32_t *D2N,
                                const uint32_t *evk, uint32_t *acc, int C, bool ntt_out, cudaStream_t st) {
        k_ks_core<LOGN, RKS><<<dim3(n + c->K, C), CoreKs::T, SMEM_KS, st>>>(
            D, D2N, evk, acc, n, ntt_out ? 1 : 0, modup_pre(c, n, D2N) != nullptr ? 1 : 0, ks_dev(c), c->d_pc,
            c->d_tw_fwd, c->d_tw_inv);
        return check_launch("k_ks_core");
    }
    static bcn_status moddown_rescale(const bcn_ctx *c, int n, const uint32_t *D, const uint32_t *acc,
                                      uint32_t *out, int C, cudaStream_t st) {
        const dim3 grid(n - 1, 2 / MD_NP, C);
        const KsDev ks = ks_dev(c);
        // the top limb's correction, shared by every limb (in place on acc's limb n-1)
        uint32_t *acc_w = const_cast<uint32_t *>(acc);
        const dim3 gtop((unsigned)((c->N / 4 + 255) / 256), 2, (unsigned)C);
        switch (c->K) {
        case 1: k_md_top<1><<<gtop, 256, 0, st>>>(acc_w, n, c->N, ks, c->d_pc); break;
        case 2: k_md_top<2><<<gtop, 256, 0, st>>>(acc_w, n, c->N, ks, c->d_pc); break;
        case 3: k_md_top<3><<<gtop, 256, 0, st>>>(acc_w, n, c->N, ks, c->d_pc); break;
        case 4: k_md_top<4><<<gtop, 256, 0, st>>>(acc_w, n, c->N, ks, c->d_pc); break;
        default: return fail(BCN_E_INVAL, "ModDown: 1 to 4 special primes");
        }
        BCN_TRY(check_launch("k_md_top"));
        switch (c->K) {
        case 1: k_md_limb<LOGN, RMD, MD_NP, 1><<<grid, CoreMd::T, SMEM_MD, st>>>(D, acc, out, n, ks, c->d_pc, c->d_tw_fwd); break;
        case 2: k_md_limb<LOGN, RMD, MD_NP, 2><<<grid, CoreMd::T, SMEM_MD, st>>>(D, acc, out, n, ks, c->d_pc, c->d_tw_fwd); break;
        case 3: k_md_limb<LOGN, RMD, MD_NP, 3><<<grid, CoreMd::T, SMEM_MD, st>>>(D, acc, out, n, ks, c->d_pc, c->d_tw_fwd); break;
        case 4: k_md_limb<LOGN, RMD, MD_NP, 4><<<grid, CoreMd::T, SMEM_MD, st>>>(D, acc, out, n, ks, c->d_pc, c->d_tw_fwd); break;
        default: return fail(BCN_E_INVAL, "ModDown: 1 to 4 special primes");
        }
        return check_launch("k_md_limb");
    }
    static bcn_status modup_hoist(const bcn_ctx *c, int n, const uint32_t *in, uint32_t *U, int C, cudaStream_t st) {
        const int dnum = (n + c->alpha - 1) / c->alpha;
        k_modup_hoist<LOGN, RKS><<<dim3(n + c->K, dnum, C), CoreKs::T, SMEM_HOIST, st>>>(in, U, n, ks_dev(c), c->d_pc,
                                                                                       c->d_tw_fwd);
        return check_launch("k_modup_hoist");
    }
    static bcn_status ks_rot(const bcn_ctx *c, int n, const uint32_t *U, const RotBatch &rb, uint32_t *acc, int C,
                             cudaStream_t st) {
        k_ks_rot<LOGN, RKS><<<dim3(n + c->K, rb.count, C), CoreKs::T, SMEM_KSROT, st>>>(U, rb, acc, n, ks_dev(c),
                                                                                     c->d_pc, c->d_tw_inv);
        return check_launch("k_ks_rot");
    }
    static bcn_status setup() {
        const int smem = (int)SMEM, smem3 = (int)SMEM3, smem_sq = (int)SMEM_SQ_NTT, smem_ks = (int)SMEM_KS;
        auto big = [](const void *k, int bytes) {
            return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess;
        };
        auto carve = [](const void *k) {
            return cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100) == cudaSuccess;
        };
        if (!big((const void *)k_ntt_fwd<LOGN, R>, smem) || !big((const void *)k_ntt_inv<LOGN, R>, smem) ||
            !big((const void *)k_square_core<LOGN, R, false>, smem3) ||
            !big((const void *)k_square_core<LOGN, R, true>, smem_sq) ||
            !big((const void *)k_ks_core<LOGN, RKS>, smem_ks) || !big((const void *)k_md_limb<LOGN, RMD, MD_NP, 1>, (int)SMEM_MD) ||
            !big((const void *)k_md_limb<LOGN, RMD, MD_NP, 2>, (int)SMEM_MD) ||
            !big((const void *)k_md_limb<LOGN, RMD, MD_NP, 3>, (int)SMEM_MD) ||
            !big((const void *)k_md_limb<LOGN, RMD, MD_NP, 4>, (int)SMEM_MD) ||
            !carve((const void *)k_square_core<LOGN, R, false>) || !carve((const void *)k_square_core<LOGN, R, true>) ||
            !carve((const void *)k_ks_core<LOGN, RKS>) || !carve((const void *)k_md_limb<LOGN, RMD, MD_NP, 1>) ||
            !carve((const void *)k_md_limb<LOGN, RMD, MD_NP, 2>) ||
            !big((const void *)k_modup_hoist<LOGN, RKS>, (int)SMEM_HOIST) ||
            !big((const void *)k_ks_rot<LOGN, RKS>, (int)SMEM_KSROT))
            return fail(BCN_E_CUDA, "cudaFuncSetAttribute failed for the NTT-based kernels");
        return BCN_OK;
    }
    static const CoreFns *fns() {
        static const CoreFns f = {&ntt, &square, &keyswitch, &moddown_rescale, &setup, &modup_hoist, &ks_rot};
        return &f;
    }
};

}  // namespace bcn
