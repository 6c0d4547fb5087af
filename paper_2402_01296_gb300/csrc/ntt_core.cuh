// Register-resident negacyclic NTT for one limb per thread block.
//
// N = 2^LOGN residues, T = N / R threads, R residues per thread.  The log N
// butterfly stages are grouped into passes of up to 4 stages (log2 R for
// R <= 16; the last pass may be shorter); inside a pass every butterfly of a
// thread pairs two of its own registers, and between passes the limb is
// re-distributed through shared memory (one padded word per 32 avoids most
// bank conflicts).
//
// Forward: Cooley-Tukey with psi merged into the twiddles (table
// psi^{brv(k)}); natural-order input, bit-reversed output.  Inverse:
// Gentleman-Sande with psi^{-brv(k)}, the passes in reverse order, then the
// N^{-1} scaling.  Stage s, butterfly group i uses table entry 2^s + i.
//
// Distribution of pass P covering stages [s0, s1): rp = s1 - s0 stages,
// stride tmin = N >> s1, G = R >> rp groups of 2^rp residues per thread;
// register u = g * 2^rp + v holds element
//     e = hi * (tmin << rp) + lo + v * tmin,
//     gidx = (tid / W) * W * G + g * W + tid mod W   (W = min(32, T)),
//     lo = gidx mod tmin,  hi = gidx / tmin.
// Only the last pass can have G > 1; there the groups of a warp interleave by
// lane, so one register across a warp is a contiguous run (coalesced NTT-domain
// loads and stores); so is one register in pass 0 (natural order: coalesced
// loads and stores of coefficient-form limbs).  Everything that selects a register is a template parameter, so the
// limb stays in registers.
//
// A pass is warp-local when every warp holds the contiguous block of 32 R
// elements [32 R w, 32 R (w + 1)): the last pass, and every pass with
// tmin <= 32.  The exchange between two warp-local passes never crosses a
// warp, so it synchronises with __syncwarp; only exchanges from or to a
// spread-out distribution (pass 0 and, for large N, pass 1) need the whole
// block.  Since every read of a spread-out distribution ends with a block
// barrier, a warp may write its own block whenever its own earlier reads are
// done; a spread-out write waits for the block unless the previous exchange of
// the same transform already ended with a block barrier.
//
// LAZY (only for q < 2^30, so 4q < 2^32): Harvey's lazy butterflies.  The
// forward transform keeps residues in [0, 4q) (input [0, 4q), output [0, 4q));
// the inverse keeps them in [0, 2q) (input [0, 2q)) and its final N^{-1}
// product returns canonical residues.  Otherwise every value stays in [0, q).
#pragma once

#include "device_math.cuh"

namespace bcn {

// A prime and the value 1 read at run time.  A lazy butterfly's addition
// written as a multiply-add by `one`, which the compiler cannot fold into a
// plain addition, issues on the FMA pipe instead of the ALU pipe; which of them
// do is the FMA bit set of NttCore (both pipes run 32-bit integer work at half
// rate, and the Shoup products already load the FMA pipe, so the best split
// is measured per kernel).  Constructed from q alone, one is the constant 1 and
// every addition stays on the ALU pipe.
struct ModQ {
    uint32_t q, one;
    __device__ __forceinline__ ModQ(uint32_t q_, uint32_t one_ = 1u) : q(q_), one(one_) {}
};

// FMA bits: which lazy-butterfly additions multiply by ModQ::one
enum : int {
    kFmaFwdMin = 1,  // forward: the subtraction of 2q under the min
    kFmaFwdSum = 2,  // forward: U + V
    kFmaInvSum = 4,  // inverse: U + V
    kFmaInvMin = 8,  // inverse: the subtraction of 2q under the min
};

template <int LOGN, int R, bool LAZY = false, int FMA = kFmaFwdMin>
struct NttCore {
    static constexpr int N = 1 << LOGN;
    static constexpr int T = N / R;
    static constexpr int LOGR = (R == 2) ? 1 : (R == 4) ? 2 : (R == 8) ? 3 : (R == 16) ? 4 : (R == 32) ? 5 : 6;
    // stages per pass: log2 R up to 4; a thread with more residues holds
    // R / 16 independent groups of 16 in every pass
    static constexpr int SP = LOGR > 4 ? 4 : LOGR;
    static constexpr int PASSES = (LOGN + SP - 1) / SP;
    static constexpr int SMEM_WORDS = N + N / 32;  // padded exchange buffer
    static constexpr int WS = T < 32 ? T : 32;     // threads of one warp
    static_assert((1 << LOGR) == R, "R must be a power of two");
    static_assert(LOGN >= LOGR, "R must not exceed N");

    __host__ __device__ static constexpr int s0_of(int p) { return p * SP; }
    __host__ __device__ static constexpr int s1_of(int p) { return (p + 1) * SP < LOGN ? (p + 1) * SP : LOGN; }
    __host__ __device__ static constexpr int rp_of(int p) { return s1_of(p) - s0_of(p); }
    static constexpr int LAST_RP = rp_of(PASSES - 1);

    // butterfly-group index of group g of thread tid in pass P
    template <int P>
    __host__ __device__ static constexpr int gidx_of(int g, int tid) {
        return (tid / WS) * WS * (R >> rp_of(P)) + g * WS + tid % WS;
    }
    // element held in register u during pass P (the defining formula)
    template <int P>
    __host__ __device__ static constexpr int elem_def(int u, int tid) {
        const int rp = rp_of(P), logtmin = LOGN - s1_of(P);
        const int g = u >> rp, v = u & ((1 << rp) - 1);
        const int gidx = gidx_of<P>(g, tid);
        const int lo = gidx & ((1 << logtmin) - 1), hi = gidx >> logtmin;
        return (hi << (logtmin + rp)) + lo + (v << logtmin);
    }
    template <int P>
    __host__ __device__ static constexpr bool warp_local() {
        // full warps only; a warp covers 32 G consecutive butterfly groups
        return T >= 32 && (T == 32 || P == PASSES - 1 || (N >> s1_of(P)) <= 32 * (R >> rp_of(P)));
    }
    __host__ __device__ static constexpr int padded(int e) { return e + (e >> 5); }
    // For every supported (LOGN, R, pass) both maps are linear in the thread:
    //   elem(u, tid)         = elem(0, tid)         + elem(u, 0)
    //   padded(elem(u, tid)) = padded(elem(0, tid)) + padded(elem(u, 0))
    // (checked exhaustively on the host), so a thread needs one base per pass
    // and every register sits at a constant offset from it.
    template <int P>
    __device__ __forceinline__ static int elem(int u, int tid) { return elem_def<P>(0, tid) + elem_def<P>(u, 0); }
    template <int P>
    __device__ __forceinline__ static int pad_base(int tid) { return padded(elem_def<P>(0, tid)); }
    template <int P>
    __host__ __device__ static constexpr int pad_off(int u) { return padded(elem_def<P>(u, 0)); }

    // Twiddle loads that the compiler may not merge with the same load of another
    // transform in the same kernel (merging keeps whole tables live in registers);
    // load_tw2 reads two consecutive entries (p 16-byte aligned).
    __device__ __forceinline__ static uint2 load_tw(const uint2 *p) {
        uint2 v;
        asm volatile("ld.global.nc.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p));
        return v;
    }
    __device__ __forceinline__ static uint4 load_tw2(const uint2 *p) {
        uint4 v;
        asm volatile("ld.global.nc.v4.u32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                     : "l"(p));
        return v;
    }
    // twiddle of butterfly group b of stage KS: entries (1 << s) + (hi << KS) + b;
    // for KS >= 1 the pair (b, b + 1), b even, is one 16-byte load
    template <int KS>
    __device__ __forceinline__ static void load_stage_tw(uint2 (&W)[1 << KS], const uint2 *tw, int s, int hi) {
        const uint2 *p = tw + (1 << s) + (hi << KS);
        if constexpr (KS == 0) {
            W[0] = load_tw(p);
        } else {
#pragma unroll
            for (int b = 0; b < (1 << KS); b += 2) {
                const uint4 v = load_tw2(p + b);
                W[b] = make_uint2(v.x, v.y);
                W[b + 1] = make_uint2(v.z, v.w);
            }
        }
    }

    // The transforms below run NP polynomials in lockstep (x[p], p < NP): they
    // share every twiddle load and every barrier, and their butterflies give the
    // scheduler NP independent streams.  Polynomial p exchanges through
    // sm + p * SMEM_WORDS.

    // FIRST: the first exchange of a transform (what ran before is unknown)
    template <int PF, int PT, bool FIRST, int NP>
    __device__ __forceinline__ static void exchange(uint32_t (&x)[NP][R], uint32_t *sm, int tid) {
        constexpr bool WF = warp_local<PF>(), WT = warp_local<PT>();
        if constexpr (FIRST && !WF) __syncthreads();
#pragma unroll
        for (int p = 0; p < NP; p++) {
            uint32_t *wf = sm + p * SMEM_WORDS + pad_base<PF>(tid);
#pragma unroll
            for (int u = 0; u < R; u++) wf[pad_off<PF>(u)] = x[p][u];
        }
        if constexpr (WF && WT)
            __syncwarp();
        else
            __syncthreads();
#pragma unroll
        for (int p = 0; p < NP; p++) {
            const uint32_t *rt = sm + p * SMEM_WORDS + pad_base<PT>(tid);
#pragma unroll
            for (int u = 0; u < R; u++) x[p][u] = rt[pad_off<PT>(u)];
        }
        if constexpr (WT)
            __syncwarp();
        else
            __syncthreads();
    }

    // stage s0 + KS of pass P (forward) for group g
    template <int P, int KS, int NP>
    __device__ __forceinline__ static void stage_fwd(uint32_t (&x)[NP][R], int g, int hi, ModQ m,
                                                     const uint2 *__restrict__ tw) {
        constexpr int rp = rp_of(P), s = s0_of(P) + KS, d = 1 << (rp - 1 - KS);
        const uint32_t q = m.q;
        uint2 Wt[1 << KS];
        load_stage_tw<KS>(Wt, tw, s, hi);
#pragma unroll
        for (int b = 0; b < (1 << KS); b++) {
            const uint2 W = Wt[b];
#pragma unroll
            for (int w = 0; w < d; w++) {
                const int u = (g << rp) + b * 2 * d + w;
#pragma unroll
                for (int p = 0; p < NP; p++) {
                    if constexpr (LAZY) {
                        const uint32_t q2 = 2 * q, nq2 = 0u - q2, xu = x[p][u];
                        const uint32_t U = min(xu, xu * ((FMA & kFmaFwdMin) ? m.one : 1u) + nq2);  // [0, 2q)
                        const uint32_t V = shoup_mul_lazy(x[p][u + d], W.x, W.y, q);
                        x[p][u] = V * ((FMA & kFmaFwdSum) ? m.one : 1u) + U;   // [0, 4q)
                        x[p][u + d] = U - V + q2;  // [0, 4q)
                    } else {
                        const uint32_t U = x[p][u], V = shoup_mul(x[p][u + d], W.x, W.y, q);
                        x[p][u] = add_mod(U, V, q);
                        x[p][u + d] = sub_mod(U, V, q);
                    }
                }
            }
        }
        if constexpr (KS + 1 < rp) stage_fwd<P, KS + 1, NP>(x, g, hi, m, tw);
    }

    // stage s0 + KS of pass P (inverse), then the stages below it
    template <int P, int KS, int NP>
    __device__ __forceinline__ static void stage_inv(uint32_t (&x)[NP][R], int g, int hi, ModQ m,
                                                     const uint2 *__restrict__ tw) {
        constexpr int rp = rp_of(P), s = s0_of(P) + KS, d = 1 << (rp - 1 - KS);
        const uint32_t q = m.q;
        uint2 Wt[1 << KS];
        load_stage_tw<KS>(Wt, tw, s, hi);
#pragma unroll
        for (int b = 0; b < (1 << KS); b++) {
            const uint2 W = Wt[b];
#pragma unroll
            for (int w = 0; w < d; w++) {
                const int u = (g << rp) + b * 2 * d + w;
#pragma unroll
                for (int p = 0; p < NP; p++) {
                    const uint32_t U = x[p][u], V = x[p][u + d];
                    if constexpr (LAZY) {
                        const uint32_t q2 = 2 * q, nq2 = 0u - q2, sum = V * ((FMA & kFmaInvSum) ? m.one : 1u) + U;
                        x[p][u] = min(sum, sum * ((FMA & kFmaInvMin) ? m.one : 1u) + nq2);                   // [0, 2q)
                        x[p][u + d] = shoup_mul_lazy(U - V + q2, W.x, W.y, q);   // [0, 2q)
                    } else {
                        x[p][u] = add_mod(U, V, q);
                        x[p][u + d] = shoup_mul(sub_mod(U, V, q), W.x, W.y, q);
                    }
                }
            }
        }
        if constexpr (KS > 0) stage_inv<P, KS - 1, NP>(x, g, hi, m, tw);
    }

    template <int P, int NP>
    __device__ __forceinline__ static void pass_fwd(uint32_t (&x)[NP][R], int tid, ModQ m,
                                                    const uint2 *__restrict__ tw) {
        constexpr int rp = rp_of(P);
#pragma unroll
        for (int g = 0; g < (R >> rp); g++) {
            const int hi = gidx_of<P>(g, tid) >> (LOGN - s1_of(P));
            stage_fwd<P, 0, NP>(x, g, hi, m, tw);
        }
    }
    template <int P, int NP>
    __device__ __forceinline__ static void pass_inv(uint32_t (&x)[NP][R], int tid, ModQ m,
                                                    const uint2 *__restrict__ tw) {
        constexpr int rp = rp_of(P);
#pragma unroll
        for (int g = 0; g < (R >> rp); g++) {
            const int hi = gidx_of<P>(g, tid) >> (LOGN - s1_of(P));
            stage_inv<P, rp - 1, NP>(x, g, hi, m, tw);
        }
    }

    template <int P, int NP>
    __device__ __forceinline__ static void forward_from(uint32_t (&x)[NP][R], uint32_t *sm, int tid, ModQ m,
                                                        const uint2 *__restrict__ tw) {
        if constexpr (P > 0) exchange<P - 1, P, P == 1, NP>(x, sm, tid);
        pass_fwd<P, NP>(x, tid, m, tw);
        if constexpr (P + 1 < PASSES) forward_from<P + 1, NP>(x, sm, tid, m, tw);
    }
    template <int P, int NP>
    __device__ __forceinline__ static void inverse_from(uint32_t (&x)[NP][R], uint32_t *sm, int tid, ModQ m,
                                                        const uint2 *__restrict__ tw) {
        pass_inv<P, NP>(x, tid, m, tw);
        if constexpr (P > 0) {
            exchange<P, P - 1, P == PASSES - 1, NP>(x, sm, tid);
            inverse_from<P - 1, NP>(x, sm, tid, m, tw);
        }
    }

    // NP polynomials: pass-0 distribution (natural order) -> last-pass
    // distribution (NTT domain); sm holds NP exchange buffers
    template <int NP>
    __device__ __forceinline__ static void forward_n(uint32_t (&x)[NP][R], uint32_t *sm, int tid, ModQ m,
                                                     const uint2 *__restrict__ tw) {
        forward_from<0, NP>(x, sm, tid, m, tw);
    }
    // NP polynomials: NTT domain -> pass-0 distribution, without the N^{-1}
    // factor; the result is canonical
    template <int NP>
    __device__ __forceinline__ static void inverse_unscaled_n(uint32_t (&x)[NP][R], uint32_t *sm, int tid, ModQ m,
                                                              const uint2 *__restrict__ tw) {
        inverse_from<PASSES - 1, NP>(x, sm, tid, m, tw);
        if constexpr (LAZY) {
#pragma unroll
            for (int p = 0; p < NP; p++)
#pragma unroll
                for (int u = 0; u < R; u++) x[p][u] = reduce_once(x[p][u], m.q);
        }
    }

    // one polynomial
    __device__ __forceinline__ static uint32_t (&as_one(uint32_t (&x)[R]))[1][R] {
        return *reinterpret_cast<uint32_t(*)[1][R]>(&x);
    }
    // x: pass-0 distribution (natural order) -> last-pass distribution (NTT domain)
    __device__ __forceinline__ static void forward(uint32_t (&x)[R], uint32_t *sm, int tid, ModQ m,
                                                   const uint2 *__restrict__ tw) {
        forward_from<0, 1>(as_one(x), sm, tid, m, tw);
    }
    // x: last-pass distribution (NTT domain) -> pass-0 distribution, times N^{-1}
    __device__ __forceinline__ static void inverse(uint32_t (&x)[R], uint32_t *sm, int tid, ModQ m,
                                                   const uint2 *__restrict__ tw, uint32_t ninv, uint32_t ninv_shoup) {
        inverse_from<PASSES - 1, 1>(as_one(x), sm, tid, m, tw);
#pragma unroll
        for (int u = 0; u < R; u++) x[u] = shoup_mul(x[u], ninv, ninv_shoup, m.q);
    }
    // the same without the N^{-1} factor (callers that folded it into their
    // inputs); the result is canonical
    __device__ __forceinline__ static void inverse_unscaled(uint32_t (&x)[R], uint32_t *sm, int tid, ModQ m,
                                                            const uint2 *__restrict__ tw) {
        inverse_unscaled_n<1>(as_one(x), sm, tid, m, tw);
    }

    // element of register u in the pass-0 distribution (natural order; one
    // register across a warp is 32 consecutive elements)
    __device__ __forceinline__ static int nat_elem(int u, int tid) { return elem<0>(u, tid); }
    // natural-order limb <-> pass-0 distribution (coalesced)
    __device__ __forceinline__ static void load_natural(uint32_t (&x)[R], const uint32_t *__restrict__ g, int tid) {
#pragma unroll
        for (int u = 0; u < R; u++) x[u] = __ldg(g + nat_elem(u, tid));
    }
    __device__ __forceinline__ static void store_natural(const uint32_t (&x)[R], uint32_t *__restrict__ g, int tid) {
#pragma unroll
        for (int u = 0; u < R; u++) g[nat_elem(u, tid)] = x[u];
    }
    // element index of register u in the NTT-domain (last-pass) distribution;
    // registers 4k..4k+3 hold 4 consecutive elements when the last pass has
    // at least 2 stages
    __device__ __forceinline__ static int ntt_elem(int u, int tid) { return elem<PASSES - 1>(u, tid); }
    static constexpr bool NTT_QUADS = LAST_RP >= 2 && R >= 4;
    // registers 2k, 2k+1 hold 2 consecutive elements
    static constexpr bool NTT_PAIRS = LAST_RP >= 1 && R >= 2;

    // NTT-domain limb <-> last-pass distribution
    __device__ __forceinline__ static void load_ntt(uint32_t (&x)[R], const uint32_t *__restrict__ g, int tid) {
        if constexpr (NTT_QUADS) {
#pragma unroll
            for (int u = 0; u < R; u += 4) {
                const uint4 v = __ldg(reinterpret_cast<const uint4 *>(g + ntt_elem(u, tid)));
                x[u] = v.x; x[u + 1] = v.y; x[u + 2] = v.z; x[u + 3] = v.w;
            }
        } else if constexpr (NTT_PAIRS) {
#pragma unroll
            for (int u = 0; u < R; u += 2) {
                const uint2 v = __ldg(reinterpret_cast<const uint2 *>(g + ntt_elem(u, tid)));
                x[u] = v.x; x[u + 1] = v.y;
            }
        } else {
#pragma unroll
            for (int u = 0; u < R; u++) x[u] = __ldg(g + ntt_elem(u, tid));
        }
    }
    __device__ __forceinline__ static void store_ntt(const uint32_t (&x)[R], uint32_t *__restrict__ g, int tid) {
        if constexpr (NTT_QUADS) {
#pragma unroll
            for (int u = 0; u < R; u += 4)
                *reinterpret_cast<uint4 *>(g + ntt_elem(u, tid)) = make_uint4(x[u], x[u + 1], x[u + 2], x[u + 3]);
        } else if constexpr (NTT_PAIRS) {
#pragma unroll
            for (int u = 0; u < R; u += 2)
                *reinterpret_cast<uint2 *>(g + ntt_elem(u, tid)) = make_uint2(x[u], x[u + 1]);
        } else {
#pragma unroll
            for (int u = 0; u < R; u++) g[ntt_elem(u, tid)] = x[u];
        }
    }
};

}  // namespace bcn
