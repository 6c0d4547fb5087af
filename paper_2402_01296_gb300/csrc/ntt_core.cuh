// Register-resident negacyclic NTT for one limb per thread block.
//
// N = 2^LOGN residues, T = N / R threads, R residues per thread.  The log N
// butterfly stages are grouped into passes of r = log2(R) stages (the last
// pass may be shorter); inside a pass every butterfly of a thread pairs two of
// its own registers, and between passes the limb is re-distributed through
// shared memory (one padded word per 32 avoids most bank conflicts).
//
// Forward: Cooley-Tukey with psi merged into the twiddles (table
// psi^{brv(k)}); natural-order input, bit-reversed output.  Inverse:
// Gentleman-Sande with psi^{-brv(k)}, the passes in reverse order, then the
// N^{-1} scaling.  Stage s, butterfly group i uses table entry 2^s + i.
//
// Distribution of pass P covering stages [s0, s1): rp = s1 - s0 stages,
// stride tmin = N >> s1, G = R >> rp groups of 2^rp residues per thread;
// register u = g * 2^rp + v holds element
//     e = hi * (tmin << rp) + lo + v * tmin,   gidx = g * T + tid,
//     lo = gidx mod tmin,  hi = gidx / tmin.
// Pass 0 is therefore e = tid + u * T (coalesced loads of natural order) and a
// full last pass gives each thread R consecutive elements.  Everything that
// selects a register is a template parameter, so the limb stays in registers.
#pragma once

#include "device_math.cuh"

namespace bcn {

template <int LOGN, int R>
struct NttCore {
    static constexpr int N = 1 << LOGN;
    static constexpr int T = N / R;
    static constexpr int LOGR = (R == 2) ? 1 : (R == 4) ? 2 : (R == 8) ? 3 : (R == 16) ? 4 : (R == 32) ? 5 : 6;
    static constexpr int PASSES = (LOGN + LOGR - 1) / LOGR;
    static constexpr int SMEM_WORDS = N + N / 32;  // padded exchange buffer
    static_assert((1 << LOGR) == R, "R must be a power of two");
    static_assert(LOGN >= LOGR, "R must not exceed N");

    __host__ __device__ static constexpr int s0_of(int p) { return p * LOGR; }
    __host__ __device__ static constexpr int s1_of(int p) { return (p + 1) * LOGR < LOGN ? (p + 1) * LOGR : LOGN; }
    __host__ __device__ static constexpr int rp_of(int p) { return s1_of(p) - s0_of(p); }
    static constexpr int LAST_RP = rp_of(PASSES - 1);

    // element held in register u during pass P
    template <int P>
    __device__ __forceinline__ static int elem(int u, int tid) {
        constexpr int rp = rp_of(P), logtmin = LOGN - s1_of(P);
        const int g = u >> rp, v = u & ((1 << rp) - 1);
        const int gidx = g * T + tid;
        const int lo = gidx & ((1 << logtmin) - 1), hi = gidx >> logtmin;
        return (hi << (logtmin + rp)) + lo + (v << logtmin);
    }
    __device__ __forceinline__ static int padded(int e) { return e + (e >> 5); }

    template <int PF, int PT>
    __device__ __forceinline__ static void exchange(uint32_t (&x)[R], uint32_t *sm, int tid) {
#pragma unroll
        for (int u = 0; u < R; u++) sm[padded(elem<PF>(u, tid))] = x[u];
        __syncthreads();
#pragma unroll
        for (int u = 0; u < R; u++) x[u] = sm[padded(elem<PT>(u, tid))];
        __syncthreads();
    }

    // stage s0 + KS of pass P (forward) for group g
    template <int P, int KS>
    __device__ __forceinline__ static void stage_fwd(uint32_t (&x)[R], int g, int hi, uint32_t q,
                                                     const uint2 *__restrict__ tw) {
        constexpr int rp = rp_of(P), s = s0_of(P) + KS, d = 1 << (rp - 1 - KS);
#pragma unroll
        for (int b = 0; b < (1 << KS); b++) {
            const uint2 W = __ldg(&tw[(1 << s) + (hi << KS) + b]);
#pragma unroll
            for (int w = 0; w < d; w++) {
                const int u = (g << rp) + b * 2 * d + w;
                const uint32_t U = x[u], V = shoup_mul(x[u + d], W.x, W.y, q);
                x[u] = add_mod(U, V, q);
                x[u + d] = sub_mod(U, V, q);
            }
        }
        if constexpr (KS + 1 < rp) stage_fwd<P, KS + 1>(x, g, hi, q, tw);
    }

    // stage s0 + KS of pass P (inverse), then the stages below it
    template <int P, int KS>
    __device__ __forceinline__ static void stage_inv(uint32_t (&x)[R], int g, int hi, uint32_t q,
                                                     const uint2 *__restrict__ tw) {
        constexpr int rp = rp_of(P), s = s0_of(P) + KS, d = 1 << (rp - 1 - KS);
#pragma unroll
        for (int b = 0; b < (1 << KS); b++) {
            const uint2 W = __ldg(&tw[(1 << s) + (hi << KS) + b]);
#pragma unroll
            for (int w = 0; w < d; w++) {
                const int u = (g << rp) + b * 2 * d + w;
                const uint32_t U = x[u], V = x[u + d];
                x[u] = add_mod(U, V, q);
                x[u + d] = shoup_mul(sub_mod(U, V, q), W.x, W.y, q);
            }
        }
        if constexpr (KS > 0) stage_inv<P, KS - 1>(x, g, hi, q, tw);
    }

    template <int P>
    __device__ __forceinline__ static void pass_fwd(uint32_t (&x)[R], int tid, uint32_t q,
                                                    const uint2 *__restrict__ tw) {
        constexpr int rp = rp_of(P);
#pragma unroll
        for (int g = 0; g < (R >> rp); g++) {
            const int hi = (g * T + tid) >> (LOGN - s1_of(P));
            stage_fwd<P, 0>(x, g, hi, q, tw);
        }
    }
    template <int P>
    __device__ __forceinline__ static void pass_inv(uint32_t (&x)[R], int tid, uint32_t q,
                                                    const uint2 *__restrict__ tw) {
        constexpr int rp = rp_of(P);
#pragma unroll
        for (int g = 0; g < (R >> rp); g++) {
            const int hi = (g * T + tid) >> (LOGN - s1_of(P));
            stage_inv<P, rp - 1>(x, g, hi, q, tw);
        }
    }

    template <int P>
    __device__ __forceinline__ static void forward_from(uint32_t (&x)[R], uint32_t *sm, int tid, uint32_t q,
                                                        const uint2 *__restrict__ tw) {
        if constexpr (P > 0) exchange<P - 1, P>(x, sm, tid);
        pass_fwd<P>(x, tid, q, tw);
        if constexpr (P + 1 < PASSES) forward_from<P + 1>(x, sm, tid, q, tw);
    }
    template <int P>
    __device__ __forceinline__ static void inverse_from(uint32_t (&x)[R], uint32_t *sm, int tid, uint32_t q,
                                                        const uint2 *__restrict__ tw) {
        pass_inv<P>(x, tid, q, tw);
        if constexpr (P > 0) {
            exchange<P, P - 1>(x, sm, tid);
            inverse_from<P - 1>(x, sm, tid, q, tw);
        }
    }

    // x: pass-0 distribution (natural order) -> last-pass distribution (NTT domain)
    __device__ __forceinline__ static void forward(uint32_t (&x)[R], uint32_t *sm, int tid, uint32_t q,
                                                   const uint2 *__restrict__ tw) {
        forward_from<0>(x, sm, tid, q, tw);
    }

    // x: last-pass distribution (NTT domain) -> pass-0 distribution, times N^{-1}
    __device__ __forceinline__ static void inverse(uint32_t (&x)[R], uint32_t *sm, int tid, uint32_t q,
                                                   const uint2 *__restrict__ tw, uint32_t ninv, uint32_t ninv_shoup) {
        inverse_from<PASSES - 1>(x, sm, tid, q, tw);
#pragma unroll
        for (int u = 0; u < R; u++) x[u] = shoup_mul(x[u], ninv, ninv_shoup, q);
    }

    // natural-order limb <-> pass-0 distribution (coalesced)
    __device__ __forceinline__ static void load_natural(uint32_t (&x)[R], const uint32_t *__restrict__ g, int tid) {
#pragma unroll
        for (int u = 0; u < R; u++) x[u] = __ldg(g + tid + u * T);
    }
    __device__ __forceinline__ static void store_natural(const uint32_t (&x)[R], uint32_t *__restrict__ g, int tid) {
#pragma unroll
        for (int u = 0; u < R; u++) g[tid + u * T] = x[u];
    }
    // element index of register u in the NTT-domain (last-pass) distribution;
    // registers 4k..4k+3 hold 4 consecutive elements when the last pass has
    // at least 2 stages
    __device__ __forceinline__ static int ntt_elem(int u, int tid) { return elem<PASSES - 1>(u, tid); }
    static constexpr bool NTT_QUADS = LAST_RP >= 2 && R >= 4;

    // NTT-domain limb <-> last-pass distribution
    __device__ __forceinline__ static void load_ntt(uint32_t (&x)[R], const uint32_t *__restrict__ g, int tid) {
        if constexpr (NTT_QUADS) {
#pragma unroll
            for (int u = 0; u < R; u += 4) {
                const uint4 v = __ldg(reinterpret_cast<const uint4 *>(g + ntt_elem(u, tid)));
                x[u] = v.x; x[u + 1] = v.y; x[u + 2] = v.z; x[u + 3] = v.w;
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
        } else {
#pragma unroll
            for (int u = 0; u < R; u++) g[ntt_elem(u, tid)] = x[u];
        }
    }
};

}  // namespace bcn
