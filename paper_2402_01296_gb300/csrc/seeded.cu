// Compact uploads.  Integer plaintexts: a plaintext whose coefficients are
// below 2^63 in magnitude travels as those integers (8 bytes a coefficient
// instead of 4 per prime) and the device reduces them mod each prime.
//
// Seeded ciphertexts: the second polynomial of a secret-key ciphertext,
// c1 = a, is uniform noise the client draws from a seed, so the client can
// send c0 and the seed instead of (c0, c1) and the server draws the same a
// (half the upload; the paper's client/server split of Sec. 2 sends every
// encrypted segment to the server).
//
// The draws follow the library's sampling: SplitMix64 (Steele, Lea, Flood
// 2014) with the stream of (seed, tag 4, index ct * 256 + limb) starting at
// mix64(seed + G ((4 << 40) + index + 1)); draw k is mix64(start + (k+1) G);
// coefficient j of limb i is the j-th draw whose low 32 bits w fall below
// floor(2^32 / q_i) q_i, reduced mod q_i.  Every draw is computed from its
// counter alone, so a block takes 512 draws at a time, keeps the accepted
// ones in order with a block-wide prefix count, and stops once N are kept.
#include <algorithm>
#include <cuda_runtime.h>

#include "device_api.h"
#include "device_math.cuh"

namespace bcn {
namespace {

constexpr uint64_t kG = 0x9E3779B97F4A7C15ull;  // SplitMix64's increment
constexpr uint64_t kTagEncA = 4;
constexpr int kThreads = 512;
constexpr uint32_t kStatusDraws = 8u;  // status bit: a limb ran out of its draw budget

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// cts [n_ct][2][level][N]: c1 of ciphertext ct (stream index (ct_base + ct) * 256
// + limb) drawn into slot 1; slot 0 is left as it is.  grid (level, n_ct).
__global__ void __launch_bounds__(kThreads) k_expand_c1(uint32_t *__restrict__ cts, int level, int N, uint64_t seed,
                                                        int ct_base, const PrimeConst *__restrict__ pc,
                                                        uint32_t *__restrict__ status) {
    __shared__ int warp_count[kThreads / 32];
    __shared__ int kept;
    const int i = blockIdx.x, ct = blockIdx.y, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t q = pc[i].q;
    const uint64_t bound = ((1ull << 32) / q) * q;
    const uint64_t index = (uint64_t)(ct_base + ct) * 256 + (uint64_t)i;
    const uint64_t start = mix64(seed + kG * ((kTagEncA << 40) + index + 1));
    uint32_t *c1 = cts + (((size_t)ct * 2 + 1) * level + i) * N;
    if (tid == 0) kept = 0;
    __syncthreads();
    // about 1 draw in 30000 is rejected for q near 2^30: N + 16384 draws are
    // far more than a limb ever needs; running out sets a status bit
    const int max_rounds = (N + 16384) / kThreads;
    for (int r = 0; r < max_rounds; r++) {
        const uint64_t k = (uint64_t)r * kThreads + tid;
        const uint64_t w = mix64(start + (k + 1) * kG) & 0xFFFFFFFFull;
        const bool ok = w < bound;
        const unsigned ballot = __ballot_sync(0xFFFFFFFFu, ok);
        if (lane == 0) warp_count[warp] = __popc(ballot);
        __syncthreads();
        int before = kept, total = 0;
        for (int v = 0; v < kThreads / 32; v++) {
            if (v < warp) before += warp_count[v];
            total += warp_count[v];
        }
        const int pos = before + __popc(ballot & ((1u << lane) - 1u));
        if (ok && pos < N) c1[pos] = (uint32_t)w % q;
        __syncthreads();  // every thread has read kept and warp_count
        if (tid == 0) kept += total;
        __syncthreads();
        if (kept >= N) return;
    }
    if (tid == 0) atomicOr(status, kStatusDraws);
}

// plaintexts given as their integer coefficients (|m| < 2^63): coeffs [n][N]
// -> pts [n][level][N], m mod q_i.  grid (ceil(N / 256), n)
__global__ void __launch_bounds__(256) k_expand_i64(const int64_t *__restrict__ coeffs, uint32_t *__restrict__ pts,
                                                    int level, int N, const PrimeConst *__restrict__ pc) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    const int v = blockIdx.y;
    const int64_t m = __ldg(reinterpret_cast<const long long *>(coeffs) + (size_t)v * N + j);
    const uint64_t a = m < 0 ? (uint64_t)0 - (uint64_t)m : (uint64_t)m;
    uint32_t *out = pts + (size_t)v * level * N + j;
    for (int i = 0; i < level; i++) {
        const uint32_t q = pc[i].q, r = barrett_reduce64(a, q, pc[i].barrett);
        out[(size_t)i * N] = m < 0 && r != 0 ? q - r : r;
    }
}

}  // namespace

bcn_status launch_expand_i64(const bcn_ctx *c, const int64_t *coeffs, int n, int level, uint32_t *pts,
                             cudaStream_t st) {
    if (n <= 0) return BCN_OK;
    if (n > 65535) return fail(BCN_E_INVAL, "integer plaintexts: more than 65535 in one call");
    k_expand_i64<<<dim3((unsigned)((c->N + 255) / 256), (unsigned)n), 256, 0, st>>>(coeffs, pts, level, c->N,
                                                                                   c->d_pc);
    return check_launch("k_expand_i64");
}

bcn_status launch_expand_c1(const bcn_ctx *c, uint32_t *cts, int n_ct, int level, uint64_t seed, int ct_base,
                            cudaStream_t st) {
    if (n_ct <= 0) return BCN_OK;
    if (n_ct > 65535) return fail(BCN_E_INVAL, "seeded ciphertexts: more than 65535 in one call");
    k_expand_c1<<<dim3((unsigned)level, (unsigned)n_ct), kThreads, 0, st>>>(cts, level, c->N, seed, ct_base, c->d_pc,
                                                                           c->d_status);
    return check_launch("k_expand_c1");
}

}  // namespace bcn

using namespace bcn;

extern "C" bcn_status bcn_expand_seeded(const bcn_ctx *c, const uint32_t *c0_dev, int n_ct, int level, uint64_t seed,
                                        int ct_base, uint32_t *cts_dev, void *stream) {
    if (!c || c->device < 0) return fail(BCN_E_INVAL, "bcn_expand_seeded: no device context");
    if (level < 1 || level > c->L || n_ct < 0 || ct_base < 0) return fail(BCN_E_INVAL, "bcn_expand_seeded: bad level or count");
    if (n_ct == 0) return BCN_OK;
    if (!c0_dev || !cts_dev || ((uintptr_t)c0_dev & 15) || ((uintptr_t)cts_dev & 15))
        return fail(BCN_E_INVAL, "bcn_expand_seeded: null or unaligned buffer");
    const size_t poly = (size_t)level * c->N, n = (size_t)n_ct;
    const uint32_t *c0_end = c0_dev + n * poly, *out_end = cts_dev + 2 * n * poly;
    if (c0_dev < out_end && cts_dev < c0_end) return fail(BCN_E_INVAL, "bcn_expand_seeded: buffers overlap");
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpy2DAsync(cts_dev, 2 * poly * 4, c0_dev, poly * 4, poly * 4, n, cudaMemcpyDeviceToDevice, st) !=
        cudaSuccess)
        return fail(BCN_E_CUDA, "bcn_expand_seeded: copy of c0 failed");
    return launch_expand_c1(c, cts_dev, n_ct, level, seed, ct_base, st);
}

extern "C" bcn_status bcn_expand_i64(const bcn_ctx *c, const int64_t *coeffs_dev, int n, int level, uint32_t *pts_dev,
                                     void *stream) {
    if (!c || c->device < 0) return fail(BCN_E_INVAL, "bcn_expand_i64: no device context");
    if (level < 1 || level > c->L || n < 0) return fail(BCN_E_INVAL, "bcn_expand_i64: bad level or count");
    if (n == 0) return BCN_OK;
    if (!coeffs_dev || !pts_dev || ((uintptr_t)coeffs_dev & 15) || ((uintptr_t)pts_dev & 15))
        return fail(BCN_E_INVAL, "bcn_expand_i64: null or unaligned buffer");
    const char *a0 = reinterpret_cast<const char *>(coeffs_dev), *a1 = a0 + (size_t)n * c->N * 8;
    const char *b0 = reinterpret_cast<const char *>(pts_dev), *b1 = b0 + (size_t)n * level * c->N * 4;
    if (a0 < b1 && b0 < a1) return fail(BCN_E_INVAL, "bcn_expand_i64: buffers overlap");
    for (int v0 = 0; v0 < n; v0 += 65535)
        BCN_TRY(launch_expand_i64(c, coeffs_dev + (size_t)v0 * c->N, std::min(65535, n - v0), level,
                                  pts_dev + (size_t)v0 * level * c->N, (cudaStream_t)stream));
    return BCN_OK;
}
