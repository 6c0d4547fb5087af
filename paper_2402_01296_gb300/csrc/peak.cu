// Integer-issue microbenchmark: the ceiling against which the NTT-based
// kernels' arithmetic is reported.
//
// Every thread of a full-occupancy grid keeps 16 words in registers and runs
// `iters` rounds of one instruction sequence on them, with no memory traffic
// beyond what the sequence itself reads (the butterflies' twiddle loads, from
// a 16-entry table that stays in L1).  Kinds:
//   0  32-bit multiply-add, low half        16 independent chains  (IMAD)
//   1  32-bit multiply-add, high half       16 independent chains  (IMAD.HI)
//   2  addition then min(y, y - q)          16 independent chains  (the conditional
//                                            subtraction every modular addition uses)
//   3  lazy forward butterflies             the NTT core's own pass code (4 stages of a
//                                            16-point transform: 32 butterflies a round)
//   4  lazy inverse butterflies             the same for the inverse transform
//   5  lazy Montgomery multiply-add         the key switch's running-sum step
//                                            (product, addition, min), 16 a round
//   6  Shoup multiply-add by a constant     the basis conversions' step (shoup_mul,
//                                            add_mod), 16 a round
//   7  signed 32 x 32 -> 64 multiply-add    16 independent chains (IMAD.WIDE: the
//                                            CUDA-core MAC's inner step)
//   8  4-way int8 x uint8 dot product       16 independent chains (dp4a)
// Kinds 3-6 use the exact device functions of the evaluator (NttCore's passes
// with the key switch's FMA-pipe choice, mont_mul_lazy, shoup_mul), so their rates are
// what the NTT-based kernels could reach with their data in registers and no
// exchange, load or barrier: the roofline their algorithmic operations are
// measured against.  Values are not meaningful; a final word per thread is
// stored only when it equals an improbable run-time value, which keeps the
// compiler from dropping the work.
#include <cuda_runtime.h>

#include "device_api.h"
#include "ntt_core.cuh"

namespace bcn {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kPeakRegs = 16;

// twiddles of the 16-point passes (any values: only the instruction stream matters)
__device__ __align__(16) uint2 g_peak_tw[16] = {
    {0x1d3a5f01u, 0x3b74be02u}, {0x0a1b2c03u, 0x14365806u}, {0x2c0ffee5u, 0x581ffdcau}, {0x13579bdfu, 0x26af37beu},
    {0x02468aceu, 0x048d159cu}, {0x1f2e3d4cu, 0x3e5c7a98u}, {0x0badc0deu, 0x175b81bcu}, {0x1234abcdu, 0x2469579au},
    {0x0fedcba9u, 0x1fdb9752u}, {0x1a2b3c4du, 0x3456789au}, {0x05a5a5a5u, 0x0b4b4b4au}, {0x1c3c5c7cu, 0x3878b8f8u},
    {0x0e0d0c0bu, 0x1c1a1816u}, {0x1b1d1f21u, 0x363a3e42u}, {0x0706050au, 0x0e0c0a14u}, {0x11223344u, 0x22446688u}};

template <int KIND>
__global__ void __launch_bounds__(kPeakThreads) k_int_peak(uint32_t *__restrict__ sink, int iters, uint32_t q,
                                                           uint32_t one, uint32_t a, uint32_t b, uint32_t qneg_inv,
                                                           uint32_t magic) {
    using C = NttCore<4, kPeakRegs, true, kFmaFwdMin | kFmaInvMin>;  // the key switch's FMA-pipe choice
    uint32_t x[kPeakRegs];
    const uint32_t seed = (blockIdx.x * kPeakThreads + threadIdx.x) * 0x9E3779B9u;
#pragma unroll
    for (int u = 0; u < kPeakRegs; u++) x[u] = (seed + (uint32_t)u * 0x85EBCA6Bu) % q;
    uint32_t k[kPeakRegs], kp[kPeakRegs];  // key words (kind 5), constants and their Shoup companions (kind 6)
#pragma unroll
    for (int u = 0; u < kPeakRegs; u++) {
        k[u] = (seed ^ ((uint32_t)u * 0xC2B2AE35u)) % q;
        kp[u] = (uint32_t)(((uint64_t)k[u] << 32) / q);
    }
    uint32_t xs = seed % q;
    long long acc64[KIND == 7 ? kPeakRegs : 1];
#pragma unroll
    for (int u = 0; u < (KIND == 7 ? kPeakRegs : 1); u++) acc64[u] = (long long)seed * (u + 1);
    const ModQ m(q, one);
#pragma unroll 1
    for (int it = 0; it < iters; it++) {
        if constexpr (KIND == 0) {
#pragma unroll
            for (int u = 0; u < kPeakRegs; u++) x[u] = x[u] * a + (b + (uint32_t)u);
        } else if constexpr (KIND == 1) {
#pragma unroll
            for (int u = 0; u < kPeakRegs; u++)
                asm volatile("mad.hi.u32 %0, %0, %1, %2;" : "+r"(x[u]) : "r"(a), "r"(b + (uint32_t)u));
        } else if constexpr (KIND == 2) {
#pragma unroll
            for (int u = 0; u < kPeakRegs; u++) x[u] = reduce_once(x[u] + a, q);
        } else if constexpr (KIND == 3) {
            uint32_t(&xx)[1][kPeakRegs] = *reinterpret_cast<uint32_t(*)[1][kPeakRegs]>(&x);
            C::template pass_fwd<0, 1>(xx, 0, m, g_peak_tw);
        } else if constexpr (KIND == 4) {
            uint32_t(&xx)[1][kPeakRegs] = *reinterpret_cast<uint32_t(*)[1][kPeakRegs]>(&x);
            C::template pass_inv<0, 1>(xx, 0, m, g_peak_tw);
        } else if constexpr (KIND == 5) {
            const uint32_t nq2 = 0u - 2 * q;
#pragma unroll
            for (int u = 0; u < kPeakRegs; u++) {
                const uint32_t s = mont_mul_lazy(xs, k[u], q, qneg_inv) + x[u];
                x[u] = min(s, s + nq2);
            }
            xs = x[kPeakRegs - 1];  // the next round multiplies the last sum (no dynamic register index)
        } else if constexpr (KIND == 6) {
#pragma unroll
            for (int u = 0; u < kPeakRegs; u++) x[u] = add_mod(x[u], shoup_mul(xs, k[u], kp[u], q), q);
            xs = x[kPeakRegs - 1];
        } else if constexpr (KIND == 7) {
#pragma unroll
            for (int u = 0; u < kPeakRegs; u++) acc64[u] += (long long)(int)a * (int)(x[u] + (uint32_t)u);
        } else {
#pragma unroll
            for (int u = 0; u < kPeakRegs; u++)  // signed weights x unsigned bytes, as a byte-plane MAC would use it
                asm volatile("dp4a.s32.u32 %0, %1, %2, %0;" : "+r"(x[u]) : "r"(a), "r"(k[u] ^ (uint32_t)it));
        }
    }
    if constexpr (KIND == 7) {
#pragma unroll
        for (int u = 0; u < kPeakRegs; u++) x[u] ^= (uint32_t)acc64[u] ^ (uint32_t)(acc64[u] >> 32);
    }
    uint32_t v = xs;
#pragma unroll
    for (int u = 0; u < kPeakRegs; u++) v ^= x[u];
    if (v == magic) sink[blockIdx.x] = v;
}

template <int KIND>
bcn_status peak_grid(int *grid) {
    int dev = 0, sms = 0, nb = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_int_peak<KIND>, kPeakThreads, 0) != cudaSuccess)
        return fail(BCN_E_CUDA, "int peak: device query failed");
    *grid = sms * (nb < 1 ? 1 : nb);
    return BCN_OK;
}

// operations one thread performs per round
constexpr double kUnitsPerRound[9] = {kPeakRegs, kPeakRegs, kPeakRegs, 32, 32, kPeakRegs, kPeakRegs,
                                      kPeakRegs, kPeakRegs};

}  // namespace
}  // namespace bcn

using namespace bcn;

extern "C" {

bcn_status bcn_int_peak_grid(int kind, int *blocks) {
    if (!blocks) return fail(BCN_E_INVAL, "bcn_int_peak_grid: null argument");
    switch (kind) {
    case 0: return peak_grid<0>(blocks);
    case 1: return peak_grid<1>(blocks);
    case 2: return peak_grid<2>(blocks);
    case 3: return peak_grid<3>(blocks);
    case 4: return peak_grid<4>(blocks);
    case 5: return peak_grid<5>(blocks);
    case 6: return peak_grid<6>(blocks);
    case 7: return peak_grid<7>(blocks);
    case 8: return peak_grid<8>(blocks);
    default: return fail(BCN_E_INVAL, "bcn_int_peak_grid: kind must be 0..8");
    }
}

bcn_status bcn_int_peak_launch(int kind, int iters, uint32_t *sink_dev, size_t sink_words, void *stream,
                               double *units_out) {
    if (!sink_dev || !units_out || iters < 1) return fail(BCN_E_INVAL, "bcn_int_peak_launch: bad argument");
    int grid = 0;
    bcn_status s = bcn_int_peak_grid(kind, &grid);
    if (s != BCN_OK) return s;
    if ((size_t)grid > sink_words) return fail(BCN_E_BUDGET, "bcn_int_peak_launch: sink smaller than the grid");
    // a data prime's constants (q < 2^30, -q^-1 mod 2^32): the values only keep
    // the arithmetic in the ranges the evaluator sees
    const uint32_t q = 1073479681u;
    uint32_t qinv = 1;
    for (int i = 0; i < 5; i++) qinv *= 2u - q * qinv;  // Newton: q * qinv = 1 mod 2^32
    const uint32_t qneg_inv = 0u - qinv;
    cudaStream_t st = (cudaStream_t)stream;
    const uint32_t a = 0x9E3779B1u, b = 0x7F4A7C15u, magic = 0xFFFFFFFFu;
    switch (kind) {
    case 0: k_int_peak<0><<<grid, kPeakThreads, 0, st>>>(sink_dev, iters, q, 1u, a, b, qneg_inv, magic); break;
    case 1: k_int_peak<1><<<grid, kPeakThreads, 0, st>>>(sink_dev, iters, q, 1u, a, b, qneg_inv, magic); break;
    case 2: k_int_peak<2><<<grid, kPeakThreads, 0, st>>>(sink_dev, iters, q, 1u, a, b, qneg_inv, magic); break;
    case 3: k_int_peak<3><<<grid, kPeakThreads, 0, st>>>(sink_dev, iters, q, 1u, a, b, qneg_inv, magic); break;
    case 4: k_int_peak<4><<<grid, kPeakThreads, 0, st>>>(sink_dev, iters, q, 1u, a, b, qneg_inv, magic); break;
    case 5: k_int_peak<5><<<grid, kPeakThreads, 0, st>>>(sink_dev, iters, q, 1u, a, b, qneg_inv, magic); break;
    case 6: k_int_peak<6><<<grid, kPeakThreads, 0, st>>>(sink_dev, iters, q, 1u, a, b, qneg_inv, magic); break;
    case 7: k_int_peak<7><<<grid, kPeakThreads, 0, st>>>(sink_dev, iters, q, 1u, a, b, qneg_inv, magic); break;
    default: k_int_peak<8><<<grid, kPeakThreads, 0, st>>>(sink_dev, iters, q, 1u, a, b, qneg_inv, magic); break;
    }
    s = check_launch("k_int_peak");
    if (s != BCN_OK) return s;
    *units_out = (double)grid * kPeakThreads * iters * kUnitsPerRound[kind];
    return BCN_OK;
}

}  // extern "C"
