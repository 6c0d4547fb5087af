// Ciphertext-branch evaluation on the device (the hot path).
//
// Per layer of the ciphertext branch (Sec. 3.2 and App. B of the paper):
//   1. MAC      out[o] = sum_t w[o][t] * in[idx[o][t]]  (integer weights, exact)
//   2. add      c0 += pt[o]                             (unidirectional connection)
//   3. square   (c0, c1) -> (c0^2, 2 c0 c1, c1^2)        (tensor square, NTT domain)
//   4. relin    key switching of c1^2: ModUp (digit decomposition + fast
//               basis conversion), inner product with the evaluation key,
//               ModDown by P
//   5. rescale  divide by the last live prime
// Steps 3-5 run over chunks of output ciphertexts whose intermediates fit in L2.
// From the first square layer on the ciphertexts stay in the NTT domain: the
// square kernel takes them there, ModDown and rescale return them there, the
// MAC and the feature add are linear; the outputs return to coefficient form.
#include <algorithm>
#include <cstdio>
#include <cuda_runtime.h>

#include "device_api.h"
#include "device_math.cuh"

namespace bcn {

// taps whose weights and indices a MAC block holds in shared memory at a time
constexpr int kMacTapChunk = 2048;
// input staging of the grouped MAC: every thread streams its taps' words
// through a private ring of kMacS stages x kMacU taps in shared memory
// (cp.async), so the loads of kMacS - 1 stages are in flight while it
// multiplies the current one
constexpr int kMacU = 4, kMacS = 3, kMacThreads = 256;
constexpr size_t kMacRingBytes = (size_t)kMacS * kMacU * kMacThreads * 16;

__device__ __forceinline__ void mac_cp_async16(uint32_t dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}

// shared memory of a grouped-MAC block with OT outputs per thread and taps
// chunks of kca: input ring, then weights [kca][OTP], then tap inputs [kca]
__host__ __device__ constexpr size_t mac_grouped_smem(int OT, int kca) {
    return kMacRingBytes + (size_t)kca * 4 * (1 + (OT + 3) / 4 * 4);
}

// ------------------------------------------------------------------- kernels
// Integer-weight MAC + feature add over output groups.  A group is a set of
// outputs that read the same taps (a conv position with all its output
// channels; a whole dense layer); each thread keeps OT outputs x 4 columns of
// signed 64-bit sums, so every input word it loads serves OT outputs.
//   out[store(g, o)][col] = sum_t gw[g][o][t] * in[gidx[g][t]][col]  (+ pt[gout[g][o]], poly 0)
// store(g, o) is the output's natural (channel, row, column) index gout[g][o]
// when store_natural, else its group-major position (g - g_base) * n_go + o
// (the order kept between layers, so a chunk of outputs is a run of groups).
// Columns run over the (poly, limb, coefficient) words of a ciphertext.  Taps
// are taken in chunks of kca (weights and input indices in shared memory).
// grid (groups in this launch * ceil(n_go/OT), ceil(2*level*N/4/256)), 256 threads.
template <int OT>
__global__ void __launch_bounds__(kMacThreads, OT <= 5 ? 3 : 2) k_mac_grouped(const uint32_t *__restrict__ in, uint32_t *__restrict__ out,
                                                     const int32_t *__restrict__ gidx, const int8_t *__restrict__ gw,
                                                     const int32_t *__restrict__ gout, const uint32_t *__restrict__ pt,
                                                     int K, int kca, int n_go, int level, int N, int g_base,
                                                     int store_natural, int t_lo, int n_tl,
                                                     const PrimeConst *__restrict__ pc) {
    constexpr int OTP = (OT + 3) / 4 * 4;  // weight row padded to whole int4 loads
    extern __shared__ __align__(16) unsigned char smraw[];
    int32_t *sw = reinterpret_cast<int32_t *>(smraw + kMacRingBytes);  // [kca][OTP] weights (0: padding tap)
    int32_t *sidx = sw + (size_t)kca * OTP;                            // [kca] input (0: padding)
    // output tiles [t_lo, t_lo + n_tl) of every group
    // output tiles vary fastest over the grid: the blocks that run together read
    // the same columns of every input, which stay in L2 between them
    const int g = g_base + blockIdx.x / n_tl, o0 = (t_lo + (int)blockIdx.x % n_tl) * OT;
    const int no = min(OT, n_go - o0);
    const size_t cols = (size_t)2 * level * N;
    const size_t col = ((size_t)blockIdx.y * blockDim.x + threadIdx.x) * 4;
    const bool active = col < cols;
    // residues are below 2^30, so signed 32 x 32 -> 64 products are exact; the
    // sums start at the limb's offset (a multiple of q >= 2^58), which keeps
    // them positive and below 2^59 (|sum of products| < 2^57 at the 2^20-tap limit)
    const int lim = active ? (int)((col / N) % level) : 0;
    const long long off0 = (long long)pc[lim].mac_offset;
    long long acc[OT][4];
#pragma unroll
    for (int o = 0; o < OT; o++) acc[o][0] = acc[o][1] = acc[o][2] = acc[o][3] = off0;
    const uint32_t *base = in + (active ? col : 0);
    for (int t0 = 0; t0 < K; t0 += kca) {  // taps in chunks that fit shared memory
        const int KC = min(kca, K - t0);
        __syncthreads();  // the previous chunk's taps are no longer read
        for (int t = threadIdx.x; t < KC; t += blockDim.x) {
            const int src = gidx[(size_t)g * K + t0 + t];
            sidx[t] = src < 0 ? 0 : src;
        }
        for (int x = threadIdx.x; x < OTP * KC; x += blockDim.x) {
            const int t = x / OTP, o = x % OTP;
            const bool live = o < no && gidx[(size_t)g * K + t0 + t] >= 0;
            sw[x] = live ? (int32_t)gw[((size_t)g * n_go + o0 + o) * K + t0 + t] : 0;
        }
        __syncthreads();
        if (!active) continue;
        // thread-private ring: slot (stage % kMacS, k) of this thread at
        // ((slot * kMacU + k) * kMacThreads + tid) * 16 bytes; only the thread
        // that copies a word reads it, so cp.async.wait_group is the only sync
        const uint32_t ring = (uint32_t)__cvta_generic_to_shared(smraw) + threadIdx.x * 16;
        const uint4 *rr = reinterpret_cast<const uint4 *>(smraw) + threadIdx.x;
        const int nst = (KC + kMacU - 1) / kMacU;
        auto issue = [&](int s) {  // taps of stage s, one commit group (empty past the last stage)
            if (s < nst) {
                const int slot = s % kMacS;
#pragma unroll
                for (int k = 0; k < kMacU; k++) {
                    const int t = s * kMacU + k;
                    if (t < KC)
                        mac_cp_async16(ring + (uint32_t)((slot * kMacU + k) * kMacThreads * 16),
                                       base + (size_t)sidx[t] * cols);
                }
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        };
#pragma unroll
        for (int s = 0; s < kMacS - 1; s++) issue(s);
        for (int s = 0; s < nst; s++) {
            issue(s + kMacS - 1);
            asm volatile("cp.async.wait_group %0;" ::"n"(kMacS - 1) : "memory");
            const int slot = s % kMacS;
#pragma unroll
            for (int k = 0; k < kMacU; k++) {
                const int t = s * kMacU + k;
                if (t < KC) {
                    const uint4 x = rr[(slot * kMacU + k) * kMacThreads];
                    const int32_t *wr = sw + t * OTP;
#pragma unroll
                    for (int o = 0; o < OT; o++) {
                        const long long w = wr[o];
                        acc[o][0] += w * (int)x.x;
                        acc[o][1] += w * (int)x.y;
                        acc[o][2] += w * (int)x.z;
                        acc[o][3] += w * (int)x.w;
                    }
                }
            }
        }
    }
    if (!active) return;
    const int poly = (int)(col / ((size_t)level * N)), i = lim;
    const uint32_t q = pc[i].q;
    const uint64_t mu = pc[i].barrett;
    // every output's index and feature word are requested before any is used
    // (independent loads, one round trip)
    int og[OT];
    uint4 r[OT];
#pragma unroll
    for (int o = 0; o < OT; o++) {
        og[o] = o < no ? (gout != nullptr ? gout[(size_t)g * n_go + o0 + o] : g * n_go + o0 + o) : 0;
        r[o].x = reduce59((uint64_t)acc[o][0], q, mu);
        r[o].y = reduce59((uint64_t)acc[o][1], q, mu);
        r[o].z = reduce59((uint64_t)acc[o][2], q, mu);
        r[o].w = reduce59((uint64_t)acc[o][3], q, mu);
    }
    if (pt != nullptr && poly == 0) {
        uint4 p[OT];
#pragma unroll
        for (int o = 0; o < OT; o++)
            if (o < no) p[o] = __ldg(reinterpret_cast<const uint4 *>(pt + (size_t)og[o] * level * N + col));
#pragma unroll
        for (int o = 0; o < OT; o++) {
            if (o < no) {
                r[o].x = add_mod(r[o].x, p[o].x, q);
                r[o].y = add_mod(r[o].y, p[o].y, q);
                r[o].z = add_mod(r[o].z, p[o].z, q);
                r[o].w = add_mod(r[o].w, p[o].w, q);
            }
        }
    }
#pragma unroll
    for (int o = 0; o < OT; o++) {
        if (o < no) {
            const int os = store_natural ? og[o] : (g - g_base) * n_go + o0 + o;
            *reinterpret_cast<uint4 *>(out + (size_t)os * cols + col) = r[o];
        }
    }
}

// The same MAC on byte planes with dp4a: a residue x = sum_b x_b 2^{8b} (bytes
// x_b), so out = sum_b 2^{8b} sum_t w_t x_{t,b}, and each plane's sum over four
// taps at a time is one dp4a (four int8 weights against four uint8 bytes,
// exact in 32 bits while |sum| <= K 127 255 < 2^31, K <= kMacDp4aMaxTaps).  The
// four residues of a tap group are transposed into plane words with eight byte
// permutations, shared by the OT outputs.  A thread keeps 2 columns x OT
// outputs x 4 planes of 32-bit sums; the epilogue recombines the planes in 64
// bits, adds the offset that makes the sum non-negative, reduces and adds the
// feature.  The instruction is faster (dp4a 52.6 against IMAD.WIDE 29.7 per SM
// and clock, measured) but the kernel is slower than k_mac_grouped (CIFAR-shaped
// network: MAC 19.6 against 14.2 ms per evaluation; the byte transposes, twice
// the load instructions and the smaller output tiles cost more than the faster
// multiply-adds save), so it runs only when asked for (mac impl 2).  Taps in
// chunks of kca (a multiple of 4), 4 taps a ring stage.
// grid (groups in this launch * ceil(n_go/OT), ceil(2*level*N/2/256)), 256 threads.
constexpr int kMacDp4aMaxTaps = 32768;
constexpr size_t kMacDp4aRingBytes = (size_t)kMacS * 4 * kMacThreads * 8;
__host__ __device__ constexpr size_t mac_dp4a_smem(int kca) {
    return kMacDp4aRingBytes + (size_t)kca / 4 * 8 * 4 + (size_t)kca * 4;
}

__device__ __forceinline__ void mac_cp_async8(uint32_t dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}

__device__ __forceinline__ int dp4a_su(uint32_t w4, uint32_t bytes4, int acc) {
    int d;
    asm("dp4a.s32.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(w4), "r"(bytes4), "r"(acc));
    return d;
}

template <int OT>
__global__ void __launch_bounds__(kMacThreads, 2) k_mac_dp4a(const uint32_t *__restrict__ in, uint32_t *__restrict__ out,
                                                             const int32_t *__restrict__ gidx,
                                                             const int8_t *__restrict__ gw,
                                                             const int32_t *__restrict__ gout,
                                                             const uint32_t *__restrict__ pt, int K, int kca, int n_go,
                                                             int level, int N, int g_base, int store_natural, int t_lo,
                                                             int n_tl, const PrimeConst *__restrict__ pc) {
    extern __shared__ __align__(16) unsigned char smraw[];
    uint32_t *sw = reinterpret_cast<uint32_t *>(smraw + kMacDp4aRingBytes);  // [kca/4][8] packed weights
    int32_t *sidx = reinterpret_cast<int32_t *>(sw + (size_t)kca / 4 * 8);   // [kca] input (0: padding)
    const int g = g_base + blockIdx.x / n_tl, o0 = (t_lo + (int)blockIdx.x % n_tl) * OT;
    const int no = min(OT, n_go - o0);
    const size_t cols = (size_t)2 * level * N;
    const size_t col = ((size_t)blockIdx.y * blockDim.x + threadIdx.x) * 2;
    const bool active = col < cols;
    int acc[OT][2][4];
#pragma unroll
    for (int o = 0; o < OT; o++)
#pragma unroll
        for (int c = 0; c < 2; c++)
#pragma unroll
            for (int b = 0; b < 4; b++) acc[o][c][b] = 0;
    const uint32_t *base = in + (active ? col : 0);
    for (int t0 = 0; t0 < K; t0 += kca) {
        const int KC = min(kca, K - t0), KQ = (KC + 3) / 4;
        __syncthreads();  // the previous chunk's taps are no longer read
        for (int t = threadIdx.x; t < KQ * 4; t += blockDim.x) {
            const int src = t < KC ? gidx[(size_t)g * K + t0 + t] : -1;
            sidx[t] = src < 0 ? 0 : src;
        }
        for (int x = threadIdx.x; x < KQ * 8; x += blockDim.x) {
            const int q = x / 8, o = x % 8;
            uint32_t word = 0;
            if (o < no) {
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    const int t = 4 * q + j;
                    if (t < KC && gidx[(size_t)g * K + t0 + t] >= 0)
                        word |= (uint32_t)(uint8_t)gw[((size_t)g * n_go + o0 + o) * K + t0 + t] << (8 * j);
                }
            }
            sw[x] = word;
        }
        __syncthreads();
        if (!active) continue;
        // thread-private ring: slot (stage % kMacS, j) at ((slot * 4 + j) * kMacThreads + tid) * 8 bytes
        const uint32_t ring = (uint32_t)__cvta_generic_to_shared(smraw) + threadIdx.x * 8;
        const uint2 *rr = reinterpret_cast<const uint2 *>(smraw) + threadIdx.x;
        auto issue = [&](int q) {  // the 4 taps of group q, one commit group (empty past the last)
            if (q < KQ) {
                const int slot = q % kMacS;
#pragma unroll
                for (int j = 0; j < 4; j++)
                    mac_cp_async8(ring + (uint32_t)((slot * 4 + j) * kMacThreads * 8),
                                  base + (size_t)sidx[4 * q + j] * cols);
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        };
#pragma unroll
        for (int q = 0; q < kMacS - 1; q++) issue(q);
        for (int q = 0; q < KQ; q++) {
            issue(q + kMacS - 1);
            asm volatile("cp.async.wait_group %0;" ::"n"(kMacS - 1) : "memory");
            const int slot = q % kMacS;
            const uint2 x0 = rr[(slot * 4 + 0) * kMacThreads], x1 = rr[(slot * 4 + 1) * kMacThreads];
            const uint2 x2 = rr[(slot * 4 + 2) * kMacThreads], x3 = rr[(slot * 4 + 3) * kMacThreads];
            uint32_t pl[2][4];  // [column][byte plane]: byte b of taps 0..3
#pragma unroll
            for (int c = 0; c < 2; c++) {
                const uint32_t a0 = c ? x0.y : x0.x, a1 = c ? x1.y : x1.x, a2 = c ? x2.y : x2.x, a3 = c ? x3.y : x3.x;
                const uint32_t u0 = __byte_perm(a0, a1, 0x5140), u1 = __byte_perm(a0, a1, 0x7362);
                const uint32_t v0 = __byte_perm(a2, a3, 0x5140), v1 = __byte_perm(a2, a3, 0x7362);
                pl[c][0] = __byte_perm(u0, v0, 0x5410);
                pl[c][1] = __byte_perm(u0, v0, 0x7632);
                pl[c][2] = __byte_perm(u1, v1, 0x5410);
                pl[c][3] = __byte_perm(u1, v1, 0x7632);
            }
#pragma unroll
            for (int o = 0; o < OT; o++) {
                const uint32_t w = sw[q * 8 + o];
#pragma unroll
                for (int c = 0; c < 2; c++)
#pragma unroll
                    for (int b = 0; b < 4; b++) acc[o][c][b] = dp4a_su(w, pl[c][b], acc[o][c][b]);
            }
        }
    }
    if (!active) return;
    const int poly = (int)(col / ((size_t)level * N)), i = (int)((col / N) % level);
    const uint32_t q = pc[i].q;
    const uint64_t mu = pc[i].barrett;
    const long long off = (long long)pc[i].mac_offset;
    // one output at a time (the plane sums leave registers as they are used)
#pragma unroll
    for (int o = 0; o < OT; o++) {
        if (o >= no) break;
        const int og = gout != nullptr ? gout[(size_t)g * n_go + o0 + o] : g * n_go + o0 + o;
        uint2 pv = make_uint2(0, 0);
        if (pt != nullptr && poly == 0) pv = __ldg(reinterpret_cast<const uint2 *>(pt + (size_t)og * level * N + col));
        uint32_t rc[2];
#pragma unroll
        for (int c = 0; c < 2; c++) {
            const long long v = (long long)acc[o][c][0] + ((long long)acc[o][c][1] << 8) +
                                ((long long)acc[o][c][2] << 16) + ((long long)acc[o][c][3] << 24) + off;
            rc[c] = barrett_reduce64((uint64_t)v, q, mu);
        }
        const int os = store_natural ? og : (g - g_base) * n_go + o0 + o;
        *reinterpret_cast<uint2 *>(out + (size_t)os * cols + col) =
            make_uint2(add_mod(rc[0], pv.x, q), add_mod(rc[1], pv.y, q));
    }
}

// Pointwise product in the NTT domain (both operands canonical):
// data[r][k] <- data[r][k] * u[r mod level][k] mod q_{r mod level}.  grid (N/256, rows)
__global__ void __launch_bounds__(256) k_mul_ntt(uint32_t *__restrict__ data, const uint32_t *__restrict__ u,
                                                 int level, int N, const PrimeConst *__restrict__ pc) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    const int row = blockIdx.y, i = row % level;
    uint32_t *x = data + (size_t)row * N + k;
    *x = barrett_reduce64((uint64_t)*x * __ldg(u + (size_t)i * N + k), pc[i].q, pc[i].barrett);
}

// Rescale alone: in [C][2][n][N] -> out [C][2][n-1][N] (coefficient form). grid (N/256, 2, C)
__global__ void __launch_bounds__(256) k_rescale(const uint32_t *__restrict__ in, uint32_t *__restrict__ out, int n,
                                                 int N, KsDev ks, const PrimeConst *__restrict__ pc) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    const int b = blockIdx.y, ct = blockIdx.z, top = n - 1;
    const uint32_t *ib = in + ((size_t)ct * 2 + b) * n * N;
    uint32_t *ob = out + ((size_t)ct * 2 + b) * (n - 1) * N;
    const uint32_t ctop = ib[(size_t)top * N + k], qtop = pc[top].q;
    const bool neg = ctop > pc[top].half;
    for (int i = 0; i < top; i++) {
        const uint32_t q = pc[i].q;
        uint32_t v = sub_mod(ib[(size_t)i * N + k], ctop, q);
        if (neg) v = add_mod(v, qtop, q);
        const uint2 qi = ks.qtop_inv[(size_t)top * ks.L + i];
        ob[(size_t)i * N + k] = shoup_mul(v, qi.x, qi.y, q);
    }
}

// rescale of C ciphertexts (coefficient form): in [C][2][n][N] -> out [C][2][n-1][N]
bcn_status launch_rescale(const bcn_ctx *c, int n, const uint32_t *in, uint32_t *out, int C, cudaStream_t st) {
    if (C <= 0) return BCN_OK;
    k_rescale<<<dim3((unsigned)((c->N + 255) / 256), 2, (unsigned)C), 256, 0, st>>>(in, out, n, c->N, ks_dev(c),
                                                                                    c->d_pc);
    return check_launch("k_rescale");
}

// x -> x * R * N^{-1} mod q over rows of N words; row r uses prime prime_of(pm, r).
// The evaluation key in this form makes one Montgomery product per digit give
// the key product already divided by N, which the key-switching kernel's
// inverse NTT then needs no longer apply.
// rows on a special prime p_m also take Phat_m^{-1} mod p_m: the key switch's
// sums there then come out as a_m Phat_m^{-1}, the factor every ModDown
// conversion applies first (once here instead of once per ciphertext, limb and
// poly)
__global__ void k_key_form(uint32_t *__restrict__ data, int N, PrimeMap pm, int L, const uint2 *__restrict__ phat_inv,
                           const PrimeConst *__restrict__ pc) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    const int row = blockIdx.y, prime = prime_of(pm, row);
    const PrimeConst &P = pc[prime];
    uint32_t *x = data + (size_t)row * N + k;
    uint32_t v = shoup_mul(*x, P.rn, P.rn_shoup, P.q);
    if (prime >= L) v = shoup_mul(v, phat_inv[prime - L].x, phat_inv[prime - L].y, P.q);
    *x = v;
}

// ------------------------------------------------------------- host helpers
static bcn_status check_device(const bcn_ctx *c) {
    if (!c) return fail(BCN_E_INVAL, "null ctx");
    if (c->device < 0) return fail(BCN_E_INVAL, "host-only ctx (created with device < 0)");
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return fail(BCN_E_CUDA, "cudaGetDevice failed");
    if (cur != c->device)
        return fail(BCN_E_INVAL, "ctx belongs to device " + std::to_string(c->device) + ", current device is " +
                                     std::to_string(cur));
    return BCN_OK;
}

static bool aligned16(const void *p) { return ((uintptr_t)p & 15) == 0; }

static size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

// names of the kernel classes (NVTX ranges)
static const char *const kClassName[BCN_KERNEL_COUNT] = {"mac", "square", "keyswitch", "moddown_rescale"};

// CUDA-event pair around one launch when the model's profiler is on; an NVTX
// range named by the kernel class always
struct Timed {
    NvtxRange range;
    Profiler *p;
    cudaStream_t st;
    int cls;
    double bytes;
    int kernels = 1;  // launches the scope covers (the reported launch count)
    size_t e0 = 0;
    Timed(Profiler *p_, cudaStream_t st_, int cls_, double bytes_)
        : range(kClassName[cls_]), p(p_ && p_->on ? p_ : nullptr), st(st_), cls(cls_), bytes(bytes_) {
        if (p) e0 = mark();
    }
    size_t mark() {
        if (p->used == p->ev.size()) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            p->ev.push_back(e);
        }
        cudaEventRecord(p->ev[p->used], st);
        return p->used++;
    }
    ~Timed() {
        if (p) {
            size_t e1 = mark();
            p->recs.push_back({cls, e0, e1, bytes, kernels});
        }
    }
};

constexpr int kMaxMacTaps = 1 << 20;  // keeps |sum| < 2^58, the MAC offset

// key-switching chunk buffers per ciphertext at level n (words): D, D2N and ACC
// (plus the MAC output Y of the chunk for an evaluation)
static size_t chunk_words(const bcn_ctx *c, int n) { return (6 * (size_t)n + 2 * (size_t)(n + c->K)) * c->N; }
static size_t chunk_bytes(const bcn_ctx *c, int n, int chunk) {
    return align_up(3 * (size_t)n * c->N * 4 * chunk) + align_up((size_t)n * c->N * 4 * chunk) +
           align_up(2 * (size_t)(n + c->K) * c->N * 4 * chunk);
}
static size_t y_chunk_bytes(const bcn_ctx *c, int n, int chunk) { return align_up(2 * (size_t)n * c->N * 4 * chunk); }
// default ciphertexts per key-switching chunk: about 4 GiB of intermediates
// (measured on the CIFAR-shaped network: chunks of 224 ciphertexts 74.6 ms per
// evaluation, of 1024 or more 73.6 ms; the intermediates of a chunk outgrow L2
// either way, and fewer, larger launches fill the SMs better)
static int default_chunk(const bcn_ctx *c, int n, int n_ct) {
    const size_t target = 4ull << 30;
    int ch = (int)std::min<size_t>(32768, std::max<size_t>(1, target / (chunk_words(c, n) * 4)));
    return std::max(1, std::min(ch, std::max(1, n_ct)));
}

struct ChunkBufs {
    uint32_t *d, *acc, *d2n;
};
// d [chunk][3][n][N], d2n [chunk][n][N], acc [chunk][2][n+K][N]
static ChunkBufs carve_chunk(const bcn_ctx *c, int n, int chunk, char *ws) {
    ChunkBufs b;
    const size_t d_b = align_up(3 * (size_t)n * c->N * 4 * chunk), d2n_b = align_up((size_t)n * c->N * 4 * chunk);
    b.d = reinterpret_cast<uint32_t *>(ws);
    b.d2n = reinterpret_cast<uint32_t *>(ws + d_b);
    b.acc = reinterpret_cast<uint32_t *>(ws + d_b + d2n_b);
    return b;
}
// the part of a chunk's buffers from ciphertext o on
static ChunkBufs chunk_from(const bcn_ctx *c, int n, const ChunkBufs &b, int o) {
    const size_t N = c->N;
    return ChunkBufs{b.d + (size_t)o * 3 * n * N, b.acc + (size_t)o * 2 * (n + c->K) * N,
                     b.d2n + (size_t)o * n * N};
}

int ks_default_chunk(const bcn_ctx *c, int n, int n_ct) { return default_chunk(c, n, n_ct); }
void ks_carve(const bcn_ctx *c, int n, int chunk, char *ws, uint32_t **d, uint32_t **d2n, uint32_t **acc) {
    ChunkBufs b = carve_chunk(c, n, chunk, ws);
    *d = b.d;
    *d2n = b.d2n;
    *acc = b.acc;
}

// outputs per thread of the grouped MAC: at most 8 (at most 5 for the dp4a
// kernel, whose 4 byte-plane sums per output and column take more registers),
// the tiles of a group as even as possible (every tile reads all of the group's
// taps)
static int mac_grouped_tile(int n_go, int max_ot = 8) {
    const int tiles = (n_go + max_ot - 1) / max_ot;
    return (n_go + tiles - 1) / tiles;
}
constexpr int kMacDp4aMaxOt = 5;

// MAC over groups [g_base, g_base + n_groups) of a layer
static bcn_status launch_mac(const bcn_ctx *c, int level, int K, int n_groups, int n_go, const int32_t *gidx,
                             const int8_t *gw, const int32_t *gout, const uint32_t *in, const uint32_t *pt,
                             uint32_t *out, cudaStream_t st, Profiler *prof = nullptr, double alg_bytes = 0,
                             int g_base = 0, bool store_natural = true, const MacTcPlan *tc = nullptr,
                             int o_lo = 0, int o_hi = -1, bool dp4a = false) {
    if (n_groups <= 0 || n_go <= 0) return BCN_OK;
    if (K > kMaxMacTaps) return fail(BCN_E_INVAL, "MAC fan-in above 2^20");
    if (o_hi < 0) o_hi = n_go;  // outputs [o_lo, o_hi) of every group, o_lo on a tile boundary
    if (tc != nullptr && tc->w16 != nullptr) {
        Timed tm(prof, st, BCN_KERNEL_MAC, alg_bytes);
        const int t_lo = o_lo / tc->tile_out, t_hi = (o_hi + tc->tile_out - 1) / tc->tile_out;
        return launch_mac_tc(c, *tc, level, K, n_groups, n_go, gidx, gout, in, pt, out, st, g_base, store_natural,
                             t_lo, t_hi - t_lo);
    }
    const int N = c->N;
    const bool use_dp4a = K <= kMacDp4aMaxTaps && dp4a;
    const int OT = mac_grouped_tile(n_go, use_dp4a ? kMacDp4aMaxOt : 8);
    const int t_lo = o_lo / OT, n_tl = (o_hi + OT - 1) / OT - t_lo;
    const size_t cols = (size_t)2 * level * N;
    if (use_dp4a) {
        const int kca = std::min((K + 3) / 4 * 4, kMacTapChunk);
        const size_t smem = mac_dp4a_smem(kca);
        if ((cols / 2 + 255) / 256 > 65535) return fail(BCN_E_INVAL, "MAC: more than 65535 column blocks");
        Timed tm(prof, st, BCN_KERNEL_MAC, alg_bytes);
        dim3 grid((unsigned)(n_groups * n_tl), (unsigned)((cols / 2 + 255) / 256));
#define BCN_MAC4(OTV)                                                                                           \
    case OTV:                                                                                                   \
        k_mac_dp4a<OTV><<<grid, kMacThreads, smem, st>>>(in, out, gidx, gw, gout, pt, K, kca, n_go, level, N, g_base, \
                                                         store_natural ? 1 : 0, t_lo, n_tl, c->d_pc);           \
        break;
        switch (OT) { BCN_MAC4(1) BCN_MAC4(2) BCN_MAC4(3) BCN_MAC4(4) BCN_MAC4(5) }
#undef BCN_MAC4
        return check_launch("k_mac_dp4a");
    }
    const int kca = std::min(K, kMacTapChunk);
    const size_t smem = mac_grouped_smem(OT, kca);
    if ((cols / 4 + 255) / 256 > 65535) return fail(BCN_E_INVAL, "MAC: more than 65535 column blocks");
    Timed tm(prof, st, BCN_KERNEL_MAC, alg_bytes);
    dim3 grid((unsigned)(n_groups * n_tl), (unsigned)((cols / 4 + 255) / 256));
#define BCN_MAC(OTV)                                                                                          \
    case OTV:                                                                                                 \
        k_mac_grouped<OTV><<<grid, kMacThreads, smem, st>>>(in, out, gidx, gw, gout, pt, K, kca, n_go, level, N, g_base, \
                                                    store_natural ? 1 : 0, t_lo, n_tl, c->d_pc);              \
        break;
    switch (OT) { BCN_MAC(1) BCN_MAC(2) BCN_MAC(3) BCN_MAC(4) BCN_MAC(5) BCN_MAC(6) BCN_MAC(7) BCN_MAC(8) }
#undef BCN_MAC
    return check_launch("k_mac_grouped");
}

// outputs per tile of the MAC kernel a layer runs (splits fall on tile boundaries)
static int mac_out_tile(const bcn_layer_plan &p, bool use_tc, bool dp4a) {
    if (use_tc && p.tc.w16 != nullptr) return p.tc.tile_out;
    return mac_grouped_tile(p.n_go, dp4a && p.K <= kMacDp4aMaxTaps ? kMacDp4aMaxOt : 8);
}

// Square activation on a chunk of C ciphertexts: Y [C][2][n][N] (coefficient
// form) -> out [C][2][n-1][N].
static bcn_status square_chunk(const bcn_ctx *c, int n, const uint32_t *evk, const uint32_t *Y, bool in_ntt,
                               const ChunkBufs &b, int C, uint32_t *out, cudaStream_t st, Profiler *prof = nullptr,
                               const KeyTable &kt = KeyTable{}) {
    const int N = c->N, K = c->K, nb = n + K, dnum = (n + c->alpha - 1) / c->alpha;
    const double limb = (double)N * 4;
    const CoreFns *f = core_fns(c);
    if (!f) return fail(BCN_E_INVAL, "unsupported ring degree");
    {
        Timed tm(prof, st, BCN_KERNEL_SQUARE, limb * C * 6.0 * n);
        BCN_TRY(f->square(c, n, Y, b.d, b.d2n, C, in_ntt, st));
    }
    {
        Timed tm(prof, st, BCN_KERNEL_KEYSWITCH, limb * ((double)C * (n + 2 * nb) + 2.0 * dnum * nb));
        if (kt.n == 0) {
            BCN_TRY(f->keyswitch(c, n, b.d, b.d2n, evk, b.acc, C, true, st));
        } else {  // one launch per request the chunk covers, with its key
            tm.kernels = 0;
            for (int r = kt.ct_base / kt.cts_per_key; r < kt.n && r * kt.cts_per_key < kt.ct_base + C; r++) {
                const int lo = std::max(r * kt.cts_per_key, kt.ct_base) - kt.ct_base;
                const int hi = std::min((r + 1) * kt.cts_per_key, kt.ct_base + C) - kt.ct_base;
                if (hi <= lo) continue;
                const ChunkBufs sb = chunk_from(c, n, b, lo);
                BCN_TRY(f->keyswitch(c, n, sb.d, sb.d2n, kt.key[r], sb.acc, hi - lo, true, st));
                tm.kernels++;
            }
        }
    }
    Timed tm(prof, st, BCN_KERNEL_MODDOWN_RESCALE, limb * C * (2.0 * n + 2.0 * nb + 2.0 * (n - 1)));
    tm.kernels = 2;  // the top limb's correction, then the per-limb kernel
    return f->moddown_rescale(c, n, b.d, b.acc, out, C, st);
}

// Square activation of C coefficient-form ciphertexts with the intermediates in
// caller-chosen memory (d [C][3][n][N], acc [C][2][n+K][N]); out [C][2][n-1][N]
// in coefficient form.
bcn_status square_relin_rescale_chunk(const bcn_ctx *c, int n, const uint32_t *evk, const uint32_t *Y, uint32_t *d,
                                      uint32_t *acc, int C, uint32_t *out, cudaStream_t st) {
    ChunkBufs b{d, acc, nullptr};
    BCN_TRY(square_chunk(c, n, evk, Y, false, b, C, out, st));
    return launch_ntt(c, out, (size_t)C * 2 * (n - 1), PrimeMap{n - 1, n - 1, 0}, true, st);
}

// ----------------------------------------------------------- device context
bcn_status device_ctx_init(bcn_ctx *c) {
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(BCN_E_CUDA, "cudaSetDevice failed");
    const int P = c->L + c->K, N = c->N;
    if (cudaMalloc(&c->d_pc, sizeof(PrimeConst) * P) != cudaSuccess ||
        cudaMalloc(&c->d_tw_fwd, sizeof(uint2) * (size_t)P * N) != cudaSuccess ||
        cudaMalloc(&c->d_tw_inv, sizeof(uint2) * (size_t)P * N) != cudaSuccess ||
        cudaMalloc(&c->d_ks, sizeof(uint32_t) * c->ks.host.size()) != cudaSuccess ||
        cudaMalloc(&c->d_status, sizeof(uint32_t)) != cudaSuccess)
        return fail(BCN_E_NOMEM, "device allocation of the context tables failed");
    if (cudaMemset(c->d_status, 0, sizeof(uint32_t)) != cudaSuccess)
        return fail(BCN_E_CUDA, "clearing the device status word failed");
    bool ok = cudaMemcpy(c->d_pc, c->h_pc.data(), sizeof(PrimeConst) * P, cudaMemcpyHostToDevice) == cudaSuccess;
    for (int t = 0; t < P && ok; t++) {
        ok = cudaMemcpy(c->d_tw_fwd + (size_t)t * N, c->h_tw_fwd[t].data(), sizeof(uint2) * N,
                        cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(c->d_tw_inv + (size_t)t * N, c->h_tw_inv[t].data(), sizeof(uint2) * N,
                        cudaMemcpyHostToDevice) == cudaSuccess;
    }
    ok = ok && cudaMemcpy(c->d_ks, c->ks.host.data(), sizeof(uint32_t) * c->ks.host.size(),
                          cudaMemcpyHostToDevice) == cudaSuccess;
    if (!ok) return fail(BCN_E_CUDA, "upload of the context tables failed");
    BCN_TRY(cores_setup_all());
    BCN_TRY(mac_tc_setup());
    const int mac_smem = (int)mac_grouped_smem(8, kMacTapChunk);
#define BCN_MSETUP(OTV)                                                                                           \
    if (cudaFuncSetAttribute(k_mac_grouped<OTV>, cudaFuncAttributeMaxDynamicSharedMemorySize, mac_smem) !=      \
        cudaSuccess)                                                                                            \
        return fail(BCN_E_CUDA, "cudaFuncSetAttribute failed for the MAC kernel");
    BCN_MSETUP(1) BCN_MSETUP(2) BCN_MSETUP(3) BCN_MSETUP(4) BCN_MSETUP(5) BCN_MSETUP(6) BCN_MSETUP(7) BCN_MSETUP(8)
#undef BCN_MSETUP
    const int dp_smem = (int)mac_dp4a_smem(kMacTapChunk);
#define BCN_M4SETUP(OTV)                                                                                          \
    if (cudaFuncSetAttribute(k_mac_dp4a<OTV>, cudaFuncAttributeMaxDynamicSharedMemorySize, dp_smem) !=         \
        cudaSuccess)                                                                                            \
        return fail(BCN_E_CUDA, "cudaFuncSetAttribute failed for the dp4a MAC kernel");
    BCN_M4SETUP(1) BCN_M4SETUP(2) BCN_M4SETUP(3) BCN_M4SETUP(4) BCN_M4SETUP(5)
#undef BCN_M4SETUP
    return BCN_OK;
}

void device_ctx_free(bcn_ctx *c) {
    cudaFree(c->d_pc);
    cudaFree(c->d_tw_fwd);
    cudaFree(c->d_tw_inv);
    cudaFree(c->d_ks);
    cudaFree(c->d_status);
    c->d_status = nullptr;
    c->d_pc = nullptr;
    c->d_tw_fwd = c->d_tw_inv = nullptr;
    c->d_ks = nullptr;
}

}  // namespace bcn

using namespace bcn;

// ===================================================================== ABI
extern "C" {

// ------------------------------------------------------------------ model
static void model_layout(bcn_model *m) {
    const bcn_ctx *c = m->ctx;
    size_t x_bytes = 0, pt_bytes = 0;
    int max_sq_level = 0, max_sq_out = 0, max_go = 1;
    bool ntt = false;  // ciphertexts stay in the NTT domain from the first square layer on
    for (size_t l = 0; l < m->layers.size(); l++) {
        bcn_layer_plan &p = m->layers[l];
        p.in_ntt = ntt ? 1 : 0;
        if (p.add && ntt) pt_bytes += align_up((size_t)p.n_out * p.level * c->N * 4);
        ntt = ntt || p.square;
        const int lout = p.square ? p.level - 1 : p.level;
        if (p.square) {
            max_sq_level = std::max(max_sq_level, p.level);
            max_sq_out = std::max(max_sq_out, p.n_out);
            max_go = std::max(max_go, p.n_go);
        }
        if (l + 1 < m->layers.size()) x_bytes = std::max(x_bytes, (size_t)p.n_out * 2 * lout * c->N * 4);
    }
    m->ws_x_bytes = align_up(x_bytes);
    int ch = m->chunk_request > 0 ? m->chunk_request : (max_sq_level ? default_chunk(c, max_sq_level, max_sq_out) : 1);
    ch = std::max(ch, max_go);  // a chunk holds whole output groups
    m->chunk = std::max(1, std::min(ch, std::max(max_go, max_sq_out)));
    m->ws_y_bytes = max_sq_level ? y_chunk_bytes(c, max_sq_level, m->chunk) : 0;
    m->ws_chunk_bytes = max_sq_level ? chunk_bytes(c, max_sq_level, m->chunk) : 0;
    m->ws_pt_bytes = align_up(pt_bytes);
}

static bcn_status model_create(bcn_ctx *c, const bcn_layer *layers, int n_layers, int stack, bcn_model **out) {
    if (!c || !layers || !out || n_layers < 1) return fail(BCN_E_INVAL, "bcn_model_create: bad argument");
    if (stack < 1 || stack > kMaxStack) return fail(BCN_E_INVAL, "bcn_model_create_stacked: 1 to 16 requests");
    *out = nullptr;
    BCN_TRY(check_device(c));
    bcn_model *m = new bcn_model();
    m->ctx = c;
    m->stack = stack;
    int level = c->L, prev_out = -1;
    std::vector<int32_t> prev_perm;
    auto cleanup = [&](bcn_status s, const std::string &msg) {
        bcn_model_destroy(m);
        return fail(s, msg);
    };
    for (int l = 0; l < n_layers; l++) {
        const bcn_layer &L = layers[l];
        bcn_layer_plan p{};
        p.type = L.type;
        p.add = L.add != 0;
        p.square = L.square != 0;
        p.s_w = L.s_w;
        p.level = level;
        std::vector<int32_t> gidx, gout;
        std::vector<int8_t> gw;
        if (!L.w_int) return cleanup(BCN_E_INVAL, "layer " + std::to_string(l) + ": null weights");
        if (L.type == BCN_LAYER_CONV) {
            if (L.cin < 1 || L.h < 1 || L.w < 1 || L.cout < 1 || L.k < 1 || L.stride < 1 || L.pad < 0 ||
                L.h + 2 * L.pad < L.k || L.w + 2 * L.pad < L.k)
                return cleanup(BCN_E_INVAL, "layer " + std::to_string(l) + ": bad conv geometry");
            const int ho = (L.h + 2 * L.pad - L.k) / L.stride + 1, wo = (L.w + 2 * L.pad - L.k) / L.stride + 1;
            p.n_in = L.cin * L.h * L.w;
            p.n_out = L.cout * ho * wo;
            p.K = L.cin * L.k * L.k;
            // one group per output position: its taps, then every output channel
            p.n_groups = ho * wo;
            p.n_go = L.cout;
            gidx.assign((size_t)p.n_groups * p.K, -1);
            gw.assign((size_t)p.n_groups * p.n_go * p.K, 0);
            gout.resize((size_t)p.n_groups * p.n_go);
            for (int oy = 0; oy < ho; oy++)
                for (int ox = 0; ox < wo; ox++) {
                    const size_t g = (size_t)oy * wo + ox;
                    for (int ci = 0; ci < L.cin; ci++)
                        for (int ky = 0; ky < L.k; ky++)
                            for (int kx = 0; kx < L.k; kx++) {
                                const int iy = oy * L.stride - L.pad + ky, ix = ox * L.stride - L.pad + kx;
                                if (iy < 0 || iy >= L.h || ix < 0 || ix >= L.w) continue;
                                const size_t t = ((size_t)ci * L.k + ky) * L.k + kx;
                                gidx[g * p.K + t] = (ci * L.h + iy) * L.w + ix;
                                for (int co = 0; co < L.cout; co++)
                                    gw[(g * p.n_go + co) * p.K + t] =
                                        L.w_int[(((size_t)co * L.cin + ci) * L.k + ky) * L.k + kx];
                            }
                    for (int co = 0; co < L.cout; co++) gout[g * p.n_go + co] = (int)((co * ho + oy) * wo + ox);
                }
        } else if (L.type == BCN_LAYER_DENSE) {
            if (L.n_in < 1 || L.n_out < 1) return cleanup(BCN_E_INVAL, "layer " + std::to_string(l) + ": bad dense");
            p.n_in = L.n_in;
            p.n_out = L.n_out;
            p.K = L.n_in;
            p.n_groups = 1;
            p.n_go = L.n_out;
            gidx.resize(p.K);
            for (int k = 0; k < p.K; k++) gidx[k] = k;
            gw.assign(L.w_int, L.w_int + (size_t)p.n_out * p.K);
            gout.resize(p.n_out);
            for (int o = 0; o < p.n_out; o++) gout[o] = o;
        } else {
            return cleanup(BCN_E_INVAL, "layer " + std::to_string(l) + ": unknown type");
        }
        if (stack > 1) {  // the same layer for `stack` requests side by side: groups replicated, inputs and
                          // outputs of request r offset by r times the layer's counts
            const int n_in1 = p.n_in, n_out1 = p.n_out, G1 = p.n_groups;
            std::vector<int32_t> gi((size_t)stack * gidx.size()), go((size_t)stack * gout.size());
            std::vector<int8_t> gwr((size_t)stack * gw.size());
            for (int r = 0; r < stack; r++) {
                for (size_t k = 0; k < gidx.size(); k++)
                    gi[r * gidx.size() + k] = gidx[k] >= 0 ? gidx[k] + r * n_in1 : -1;
                for (size_t k = 0; k < gout.size(); k++) go[r * gout.size() + k] = gout[k] + r * n_out1;
                std::copy(gw.begin(), gw.end(), gwr.begin() + r * gw.size());
            }
            gidx.swap(gi);
            gout.swap(go);
            gw.swap(gwr);
            p.n_in *= stack;
            p.n_out *= stack;
            p.n_groups = G1 * stack;
        }
        if (p.K > kMaxMacTaps) return cleanup(BCN_E_INVAL, "layer fan-in above 2^20");
        if ((long long)p.n_groups * ((p.n_go + 7) / 8) > (1ll << 30))
            return cleanup(BCN_E_INVAL, "layer " + std::to_string(l) + ": too many output tiles");
        if (prev_out >= 0 && p.n_in != prev_out)
            return cleanup(BCN_E_INVAL, "layer " + std::to_string(l) + ": input count does not match");
        if (p.square && level < 2)
            return cleanup(BCN_E_LEVEL, "no level left for the square of layer " + std::to_string(l));
        if (p.square && l + 1 == n_layers)
            return cleanup(BCN_E_INVAL, "the last layer gives the outputs and must not square");
        if (!prev_perm.empty())  // inputs live in the previous layer's group-major order
            for (int32_t &v : gidx)
                if (v >= 0) v = prev_perm[v];
        std::vector<char> used(p.n_in, 0);
        for (int32_t v : gidx)
            if (v >= 0) used[v] = 1;
        p.n_distinct_in = 0;
        for (char u : used) p.n_distinct_in += u;
        m->layers.push_back(p);
        bcn_layer_plan &q = m->layers.back();
        if (cudaMalloc(&q.d_gidx, gidx.size() * 4) != cudaSuccess || cudaMalloc(&q.d_gw, gw.size()) != cudaSuccess ||
            cudaMalloc(&q.d_gout, gout.size() * 4) != cudaSuccess)
            return cleanup(BCN_E_NOMEM, "device allocation of layer tables failed");
        if (cudaMemcpy(q.d_gidx, gidx.data(), gidx.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(q.d_gw, gw.data(), gw.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(q.d_gout, gout.data(), gout.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess)
            return cleanup(BCN_E_CUDA, "upload of layer tables failed");
        if (mac_tc_eligible(c, q.K, q.n_go)) {
            // conv and dense weights are [n_go][K] in tap order, the same for every group
            bcn_status s = mac_tc_plan(c, q.K, q.n_go, L.w_int, &q.tc);
            if (s != BCN_OK) return cleanup(s, bcn_last_error());
        }
        if (p.square) level -= 1;
        prev_out = p.n_out;
        prev_perm.assign(p.n_out, 0);  // natural index -> group-major position
        for (size_t k = 0; k < gout.size(); k++) prev_perm[gout[k]] = (int32_t)k;
    }
    m->out_level = level;
    m->chunk_request = 0;
    model_layout(m);
    *out = m;
    return BCN_OK;
}

bcn_status bcn_model_create(bcn_ctx *c, const bcn_layer *layers, int n_layers, bcn_model **out) {
    return model_create(c, layers, n_layers, 1, out);
}

bcn_status bcn_model_create_stacked(bcn_ctx *c, const bcn_layer *layers, int n_layers, int requests,
                                    bcn_model **out) {
    return model_create(c, layers, n_layers, requests, out);
}

bcn_status bcn_model_set_chunk(bcn_model *m, int chunk) {
    if (!m) return fail(BCN_E_INVAL, "bcn_model_set_chunk: null model");
    m->chunk_request = chunk > 0 ? chunk : 0;
    model_layout(m);
    return BCN_OK;
}

bcn_status bcn_model_set_overlap(bcn_model *m, int on) {
    if (!m || on < 0 || on > 1) return fail(BCN_E_INVAL, "bcn_model_set_overlap: bad argument");
    m->overlap = on;
    return BCN_OK;
}

bcn_status bcn_model_set_mac_impl(bcn_model *m, int impl) {
    if (!m || impl < 0 || impl > 2) return fail(BCN_E_INVAL, "bcn_model_set_mac_impl: bad argument");
    m->mac_impl = impl;
    return BCN_OK;
}

// ------------------------------------------------------------ debug checks
// With a context's debug checks on (bcn_ctx_set_debug, or every context of a
// library built with -DBCN_DEBUG) the entry points check their inputs on the
// device before launching anything: a failed check sets a bit of the status
// word (never a trap), the host waits for the checks and refuses the call.
namespace {
constexpr uint32_t kStatusResidue = 2u, kStatusIndex = 4u;

// every word of polys [..][level][N] (limb i mod q_i) below its prime
__global__ void __launch_bounds__(256) k_check_residues(const uint32_t *__restrict__ a, size_t n_words, int level,
                                                        int N, const PrimeConst *__restrict__ pc,
                                                        uint32_t *__restrict__ status) {
    for (size_t w = (size_t)blockIdx.x * blockDim.x + threadIdx.x; w < n_words; w += (size_t)gridDim.x * blockDim.x)
        if (__ldg(a + w) >= pc[(w / N) % level].q) {
            atomicOr(status, kStatusResidue);
            return;
        }
}

// every entry of a table inside [lo, hi)
__global__ void __launch_bounds__(256) k_check_index(const int32_t *__restrict__ v, size_t n, int lo, int hi,
                                                     uint32_t *__restrict__ status) {
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
        if (__ldg(v + k) < lo || __ldg(v + k) >= hi) {
            atomicOr(status, kStatusIndex);
            return;
        }
}

unsigned check_grid(size_t n) { return (unsigned)std::min<size_t>((n + 255) / 256, 4096); }

// checks run only outside stream capture (a captured graph replays without them)
bool debug_on(const bcn_ctx *c, cudaStream_t st) {
    if (!c->debug) return false;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone;
}

bcn_status debug_residues(const bcn_ctx *c, const uint32_t *a, size_t n_poly, int level, cudaStream_t st) {
    const size_t n = n_poly * (size_t)level * c->N;
    if (n == 0 || !a) return BCN_OK;
    k_check_residues<<<check_grid(n), 256, 0, st>>>(a, n, level, c->N, c->d_pc, c->d_status);
    return check_launch("k_check_residues");
}

bcn_status debug_index(const bcn_ctx *c, const int32_t *v, size_t n, int lo, int hi, cudaStream_t st) {
    if (n == 0 || !v) return BCN_OK;
    k_check_index<<<check_grid(n), 256, 0, st>>>(v, n, lo, hi, c->d_status);
    return check_launch("k_check_index");
}

// wait for the checks; a set bit refuses the call (and is cleared)
bcn_status debug_outcome(const bcn_ctx *c, cudaStream_t st, const char *who) {
    uint32_t s = 0;
    if (cudaStreamSynchronize(st) != cudaSuccess || cudaMemcpy(&s, c->d_status, 4, cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(BCN_E_CUDA, std::string(who) + ": reading the debug checks failed");
    const uint32_t bad = s & (kStatusResidue | kStatusIndex);
    if (!bad) return BCN_OK;
    const uint32_t keep = s & ~bad;
    if (cudaMemcpy(c->d_status, &keep, 4, cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(BCN_E_CUDA, std::string(who) + ": clearing the debug bits failed");
    return fail(BCN_E_INVAL, std::string(who) + (bad & kStatusResidue ? ": an input residue is not below its prime"
                                                                       : ": a table index is out of range"));
}
}  // namespace

extern "C++" {
namespace bcn {
bcn_status debug_check_input(const bcn_ctx *c, const uint32_t *a, size_t n_poly, int level, cudaStream_t st,
                             const char *who) {
    if (!debug_on(c, st)) return BCN_OK;
    BCN_TRY(debug_residues(c, a, n_poly, level, st));
    return debug_outcome(c, st, who);
}
}  // namespace bcn
}

bcn_status bcn_ctx_set_debug(bcn_ctx *c, int on) {
    if (!c) return fail(BCN_E_INVAL, "bcn_ctx_set_debug: null context");
    c->debug = on != 0;
    return BCN_OK;
}

bcn_status bcn_ctx_get_debug(const bcn_ctx *c, int *on) {
    if (!c || !on) return fail(BCN_E_INVAL, "bcn_ctx_get_debug: null argument");
    *on = c->debug ? 1 : 0;
    return BCN_OK;
}

bcn_status bcn_device_status(const bcn_ctx *c, uint32_t *status) {
    if (!c || !status) return fail(BCN_E_INVAL, "bcn_device_status: null argument");
    BCN_TRY(check_device(c));
    if (cudaMemcpy(status, c->d_status, 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemset(c->d_status, 0, 4) != cudaSuccess)
        return fail(BCN_E_CUDA, "bcn_device_status: reading the status word failed");
    return BCN_OK;
}

bcn_status bcn_model_destroy(bcn_model *m) {
    if (!m) return BCN_OK;
    for (auto &p : m->layers) {
        cudaFree(p.d_gidx);
        cudaFree(p.d_gw);
        cudaFree(p.d_gout);
        cudaFree(p.tc.w16);
    }
    for (auto e : m->prof.ev) cudaEventDestroy(e);
    for (auto s2 : m->copy_streams) cudaStreamDestroy(s2);
    for (auto &kv : m->staging_free) cudaEventDestroy(kv.second);
    if (m->split_stream) cudaStreamDestroy(m->split_stream);
    if (m->aux_stream) cudaStreamDestroy(m->aux_stream);
    delete m;
    return BCN_OK;
}

bcn_status bcn_model_get_info(const bcn_model *m, bcn_model_info *o) {
    if (!m || !o) return fail(BCN_E_INVAL, "bcn_model_get_info: null argument");
    o->n_layers = (int)m->layers.size();
    o->n_in = m->layers.front().n_in;
    o->n_out = m->layers.back().n_out;
    o->out_level = m->out_level;
    o->n_add = 0;
    o->stack = m->stack;
    for (auto &p : m->layers) o->n_add += p.add;
    return BCN_OK;
}

bcn_status bcn_model_layers(const bcn_model *m, int *level_out, int *n_out_out) {
    if (!m || !level_out || !n_out_out) return fail(BCN_E_INVAL, "bcn_model_layers: null argument");
    for (size_t l = 0; l < m->layers.size(); l++) {
        level_out[l] = m->layers[l].level;
        n_out_out[l] = m->layers[l].n_out;
    }
    return BCN_OK;
}

bcn_status bcn_model_scales(const bcn_model *m, double input_scale, double *add_scales, double *out_scale) {
    if (!m || !out_scale) return fail(BCN_E_INVAL, "bcn_model_scales: null argument");
    double S = input_scale;
    int a = 0;
    for (auto &p : m->layers) {
        S = S / p.s_w;
        if (p.add) {
            if (add_scales) add_scales[a] = S;
            a++;
        }
        if (p.square) S = S * S / (double)m->ctx->primes[p.level - 1];
    }
    *out_scale = S;
    return BCN_OK;
}

bcn_status bcn_evk_prepare(const bcn_ctx *c, const uint32_t *evk, uint32_t *evk_eval, void *stream) {
    BCN_TRY(check_device(c));
    if (!evk || !evk_eval || !aligned16(evk) || !aligned16(evk_eval))
        return fail(BCN_E_INVAL, "bcn_evk_prepare: null or unaligned buffer");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t words = bcn_evk_words(c);
    if (evk != evk_eval && cudaMemcpyAsync(evk_eval, evk, words * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return fail(BCN_E_CUDA, "bcn_evk_prepare: copy failed");
    const PrimeMap all = data_map(c->L + c->K);
    const size_t rows = (size_t)c->dnum * 2 * (c->L + c->K);
    BCN_TRY(launch_ntt(c, evk_eval, rows, all, false, st));
    k_key_form<<<dim3((c->N + 255) / 256, (unsigned)rows), 256, 0, st>>>(evk_eval, c->N, all, c->L,
                                                                         ks_dev(c).phat_inv, c->d_pc);
    return check_launch("k_key_form");
}

bcn_status bcn_eval_workspace_bytes(const bcn_model *m, size_t *bytes) {
    if (!m || !bytes) return fail(BCN_E_INVAL, "bcn_eval_workspace_bytes: null argument");
    *bytes = 2 * m->ws_x_bytes + m->ws_y_bytes + m->ws_chunk_bytes + m->ws_pt_bytes;
    return BCN_OK;
}

// The evaluation; with layer_ready, the stream waits for layer_ready[l] (when
// not null) before layer l's first launch (bcn_eval_host: feature copies).
static bcn_status eval_impl(const bcn_model *m, const uint32_t *evk, const uint32_t *cts, const uint32_t *const *pts,
                            uint32_t *out, void *ws, size_t ws_bytes, void *stream,
                            const std::vector<std::vector<cudaEvent_t>> *layer_ready,
                            const uint32_t *const *keys = nullptr);

bcn_status bcn_eval_stacked(const bcn_model *m, const uint32_t *const *evk_evals, int n_keys, const uint32_t *cts,
                            const uint32_t *const *pts, uint32_t *out, void *ws, size_t ws_bytes, void *stream) {
    if (!m || !evk_evals || n_keys != m->stack) return fail(BCN_E_INVAL, "bcn_eval_stacked: one key per request");
    for (int r = 0; r < n_keys; r++)
        if (!evk_evals[r] || ((uintptr_t)evk_evals[r] & 15))
            return fail(BCN_E_INVAL, "bcn_eval_stacked: null or unaligned key");
    return eval_impl(m, evk_evals[0], cts, pts, out, ws, ws_bytes, stream, nullptr, evk_evals);
}

bcn_status bcn_eval(const bcn_model *m, const uint32_t *evk, const uint32_t *cts, const uint32_t *const *pts,
                    uint32_t *out, void *ws, size_t ws_bytes, void *stream) {
    return eval_impl(m, evk, cts, pts, out, ws, ws_bytes, stream, nullptr);
}

static bcn_status eval_impl(const bcn_model *m, const uint32_t *evk, const uint32_t *cts, const uint32_t *const *pts,
                            uint32_t *out, void *ws, size_t ws_bytes, void *stream,
                            const std::vector<std::vector<cudaEvent_t>> *layer_ready,
                            const uint32_t *const *keys) {
    if (!m) return fail(BCN_E_INVAL, "bcn_eval: null model");
    NvtxRange r_eval("bcn_eval");
    const bcn_ctx *c = m->ctx;
    BCN_TRY(check_device(c));
    size_t need = 0;
    bcn_eval_workspace_bytes(m, &need);
    if (ws_bytes < need) return fail(BCN_E_BUDGET, "bcn_eval: workspace too small");
    if (!cts || !out || (need && !ws) || !evk) return fail(BCN_E_INVAL, "bcn_eval: null buffer");
    if (!aligned16(cts) || !aligned16(out) || !aligned16(ws) || !aligned16(evk))
        return fail(BCN_E_INVAL, "bcn_eval: buffers must be 16-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    // square layers split their chunks over `st` and the model's split stream,
    // unless kernel timing is on (its events are on `st` alone)
    cudaStream_t split = nullptr;
    cudaEvent_t split_ev[2] = {nullptr, nullptr};
    struct EventPair {
        cudaEvent_t *e;
        ~EventPair() {
            for (int i = 0; i < 2; i++)
                if (e[i]) cudaEventDestroy(e[i]);
        }
    } split_guard{split_ev};
    bool has_square = false;
    for (auto &l : m->layers) has_square |= l.square != 0;
    if (!m->prof.on && m->overlap && has_square) {
        bcn_model *mm = const_cast<bcn_model *>(m);
        std::lock_guard<std::mutex> lock(mm->split_mu);
        if (!mm->split_stream && cudaStreamCreateWithFlags(&mm->split_stream, cudaStreamNonBlocking) != cudaSuccess)
            return fail(BCN_E_CUDA, "bcn_eval: stream creation failed");
        split = mm->split_stream;
        if (cudaEventCreateWithFlags(&split_ev[0], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&split_ev[1], cudaEventDisableTiming) != cudaSuccess)
            return fail(BCN_E_CUDA, "bcn_eval: event creation failed");
    }
    char *w = reinterpret_cast<char *>(ws);
    uint32_t *X[2] = {reinterpret_cast<uint32_t *>(w), reinterpret_cast<uint32_t *>(w + m->ws_x_bytes)};
    uint32_t *Ychunk = reinterpret_cast<uint32_t *>(w + 2 * m->ws_x_bytes);
    char *chunk_ws = w + 2 * m->ws_x_bytes + m->ws_y_bytes;
    // the input ciphertexts are in coefficient form; from the first square layer
    // on they stay in the NTT domain (the MAC is linear, so it runs in either),
    // and the last layer's outputs return to coefficient form at the end.  The
    // feature plaintexts that join NTT-domain ciphertexts are transformed (into
    // their own slices of the workspace) on the model's aux stream, forked from
    // `st` at the start, while the layers before them run; each such layer's MAC
    // waits for its event.  With kernel timing on they run on `st` in place.
    const size_t N = c->N;
    std::vector<uint32_t *> pt_ntt(m->layers.size(), nullptr);
    std::vector<cudaEvent_t> pt_ev(m->layers.size(), nullptr);
    struct EventList {
        std::vector<cudaEvent_t> &e;
        ~EventList() {
            for (cudaEvent_t v : e)
                if (v) cudaEventDestroy(v);
        }
    } pt_guard{pt_ev};
    {
        char *PT = chunk_ws + m->ws_chunk_bytes;
        int a = 0;
        for (size_t l = 0; l < m->layers.size(); l++) {
            const bcn_layer_plan &p = m->layers[l];
            if (!p.add) continue;
            if (!pts || !pts[a] || !aligned16(pts[a])) return fail(BCN_E_INVAL, "bcn_eval: missing feature plaintexts");
            a++;
            if (!p.in_ntt) continue;
            pt_ntt[l] = reinterpret_cast<uint32_t *>(PT);
            PT += align_up((size_t)p.n_out * p.level * N * 4);
        }
    }
    if (layer_ready == nullptr && debug_on(c, st)) {
        const bcn_layer_plan &p0 = m->layers.front();
        BCN_TRY(debug_residues(c, cts, 2 * (size_t)p0.n_in, p0.level, st));
        int a = 0;
        for (const bcn_layer_plan &p : m->layers) {
            if (p.add) BCN_TRY(debug_residues(c, pts[a++], (size_t)p.n_out, p.level, st));
            BCN_TRY(debug_index(c, p.d_gidx, (size_t)p.n_groups * p.K, -1, p.n_in, st));
            BCN_TRY(debug_index(c, p.d_gout, (size_t)p.n_groups * p.n_go, 0, p.n_out, st));
        }
        BCN_TRY(debug_outcome(c, st, "bcn_eval"));
    }
    cudaStream_t aux = nullptr;
    bool any_pt_ntt = false;
    for (uint32_t *q : pt_ntt) any_pt_ntt |= q != nullptr;
    if (!m->prof.on && m->overlap && any_pt_ntt) {
        bcn_model *mm = const_cast<bcn_model *>(m);
        {
            std::lock_guard<std::mutex> lock(mm->split_mu);
            if (!mm->aux_stream && cudaStreamCreateWithFlags(&mm->aux_stream, cudaStreamNonBlocking) != cudaSuccess)
                return fail(BCN_E_CUDA, "bcn_eval: stream creation failed");
            aux = mm->aux_stream;
        }
        cudaEvent_t fork = nullptr;
        if (cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess)
            return fail(BCN_E_CUDA, "bcn_eval: event creation failed");
        const bool forked = cudaEventRecord(fork, st) == cudaSuccess && cudaStreamWaitEvent(aux, fork, 0) == cudaSuccess;
        cudaEventDestroy(fork);
        if (!forked) return fail(BCN_E_CUDA, "bcn_eval: fork failed");
        int a = 0;
        for (size_t l = 0; l < m->layers.size(); l++) {
            const bcn_layer_plan &p = m->layers[l];
            if (!p.add) continue;
            const uint32_t *pt = pts[a++];
            if (!pt_ntt[l]) continue;
            if (layer_ready != nullptr)
                for (cudaEvent_t e : (*layer_ready)[l])
                    if (cudaStreamWaitEvent(aux, e, 0) != cudaSuccess) return fail(BCN_E_CUDA, "bcn_eval: event wait");
            const size_t bytes = (size_t)p.n_out * p.level * N * 4;
            if (cudaMemcpyAsync(pt_ntt[l], pt, bytes, cudaMemcpyDeviceToDevice, aux) != cudaSuccess)
                return fail(BCN_E_CUDA, "bcn_eval: feature copy failed");
            BCN_TRY(launch_ntt(c, pt_ntt[l], (size_t)p.n_out * p.level, data_map(p.level), false, aux));
            if (cudaEventCreateWithFlags(&pt_ev[l], cudaEventDisableTiming) != cudaSuccess ||
                cudaEventRecord(pt_ev[l], aux) != cudaSuccess)
                return fail(BCN_E_CUDA, "bcn_eval: event record failed");
        }
    }
    const uint32_t *x = cts;
    int a = 0;
    Profiler *prof = &m->prof;
    const bool dp4a = m->mac_impl == 2;  // byte-plane dp4a MAC on the CUDA cores (measured slower: opt-in)
    for (size_t l = 0; l < m->layers.size(); l++) {
        const bcn_layer_plan &p = m->layers[l];
        char lname[32];
        snprintf(lname, sizeof lname, "layer %d", (int)l);
        NvtxRange r_layer(lname);
        const bool last = l + 1 == m->layers.size();
        uint32_t *y = last ? out : X[l % 2];
        if (layer_ready != nullptr)
            for (cudaEvent_t e : (*layer_ready)[l])
                if (cudaStreamWaitEvent(st, e, 0) != cudaSuccess) return fail(BCN_E_CUDA, "bcn_eval: event wait");
        const uint32_t *pt = nullptr;
        const double limb = (double)N * 4;
        if (p.add) {
            if (!pts || !pts[a] || !aligned16(pts[a]))
                return fail(BCN_E_INVAL, "bcn_eval: missing feature plaintexts");
            pt = pts[a++];
            if (pt_ev[l] != nullptr) {  // transformed on the aux stream
                if (cudaStreamWaitEvent(st, pt_ev[l], 0) != cudaSuccess)
                    return fail(BCN_E_CUDA, "bcn_eval: event wait");
                pt = pt_ntt[l];
            } else if (pt_ntt[l] != nullptr) {  // kernel timing: on `st`
                const size_t bytes = (size_t)p.n_out * p.level * N * 4;
                Timed tm(prof, st, BCN_KERNEL_SQUARE, 2.0 * bytes);
                if (cudaMemcpyAsync(pt_ntt[l], pt, bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
                    return fail(BCN_E_CUDA, "bcn_eval: feature copy failed");
                BCN_TRY(launch_ntt(c, pt_ntt[l], (size_t)p.n_out * p.level, data_map(p.level), false, st));
                pt = pt_ntt[l];
            }
        }
        if (!p.square) {
            const double mac_bytes = limb * ((double)p.n_distinct_in * 2 * p.level + (double)p.n_out * 2 * p.level +
                                             (pt ? (double)p.n_out * p.level : 0.0));
            BCN_TRY(launch_mac(c, p.level, p.K, p.n_groups, p.n_go, p.d_gidx, p.d_gw, p.d_gout, x, pt, y, st, prof,
                               mac_bytes, 0, last, m->mac_impl == 0 ? &p.tc : nullptr, 0, -1, dp4a));
        } else {
            const int n = p.level;
            const int gpc = std::max(1, m->chunk / p.n_go);  // whole groups per chunk
            ChunkBufs b = carve_chunk(c, n, m->chunk, chunk_ws);
            const MacTcPlan *tc = m->mac_impl == 0 ? &p.tc : nullptr;
            const int ts = mac_out_tile(p, tc != nullptr, dp4a);
            for (int g0 = 0; g0 < p.n_groups; g0 += gpc) {
                const int ng = std::min(gpc, p.n_groups - g0), C = ng * p.n_go, o0 = g0 * p.n_go;
                const double mac_bytes = limb * ((double)p.n_distinct_in * 2 * n * ng / p.n_groups +
                                                 (double)C * 2 * n + (pt ? (double)C * n : 0.0));
                uint32_t *yo = y + (size_t)o0 * 2 * (n - 1) * N;
                // Two halves side by side (MAC, then square, key switch, ModDown
                // and rescale), the second on the split stream forked from and
                // joined back to `st`, each on its own slices of the chunk
                // buffers: one half's MAC overlaps the other's NTT kernels and
                // their blocks fill each other's last waves.  Halves of several
                // groups split by groups, of one group by output tiles.
                const int ngA = (ng + 1) / 2;
                const int oA = ng >= 2 ? ngA * p.n_go : std::min(p.n_go, (((p.n_go + ts - 1) / ts + 1) / 2) * ts);
                // a stacked model's ciphertext at group-major position o belongs to request
                // o / (n_out / stack) and uses that request's key
                KeyTable ktA{}, ktB{};
                if (keys != nullptr) {
                    for (int r = 0; r < m->stack; r++) ktA.key[r] = ktB.key[r] = keys[r];
                    ktA.n = ktB.n = m->stack;
                    ktA.cts_per_key = ktB.cts_per_key = p.n_out / m->stack;
                    ktA.ct_base = o0;
                    ktB.ct_base = o0 + oA;
                }
                if (split == nullptr || oA >= C) {
                    BCN_TRY(launch_mac(c, n, p.K, ng, p.n_go, p.d_gidx, p.d_gw, p.d_gout, x, pt, Ychunk, st, prof,
                                       mac_bytes, g0, false, tc, 0, -1, dp4a));
                    BCN_TRY(square_chunk(c, n, evk, Ychunk, p.in_ntt != 0, b, C, yo, st, prof, ktA));
                    continue;
                }
                const int C1 = C - oA;
                const ChunkBufs b1 = chunk_from(c, n, b, oA);
                if (cudaEventRecord(split_ev[0], st) != cudaSuccess ||
                    cudaStreamWaitEvent(split, split_ev[0], 0) != cudaSuccess)
                    return fail(BCN_E_CUDA, "bcn_eval: fork failed");
                if (ng >= 2) {
                    BCN_TRY(launch_mac(c, n, p.K, ngA, p.n_go, p.d_gidx, p.d_gw, p.d_gout, x, pt, Ychunk, st, nullptr,
                                       0, g0, false, tc, 0, -1, dp4a));
                    BCN_TRY(launch_mac(c, n, p.K, ng - ngA, p.n_go, p.d_gidx, p.d_gw, p.d_gout, x, pt,
                                       Ychunk + (size_t)oA * 2 * n * N, split, nullptr, 0, g0 + ngA, false, tc, 0, -1,
                                       dp4a));
                } else {  // one group: outputs [0, oA) and [oA, n_go), both stored at their group positions
                    BCN_TRY(launch_mac(c, n, p.K, 1, p.n_go, p.d_gidx, p.d_gw, p.d_gout, x, pt, Ychunk, st, nullptr,
                                       0, g0, false, tc, 0, oA, dp4a));
                    BCN_TRY(launch_mac(c, n, p.K, 1, p.n_go, p.d_gidx, p.d_gw, p.d_gout, x, pt, Ychunk, split, nullptr,
                                       0, g0, false, tc, oA, p.n_go, dp4a));
                }
                BCN_TRY(square_chunk(c, n, evk, Ychunk, p.in_ntt != 0, b, oA, yo, st, nullptr, ktA));
                BCN_TRY(square_chunk(c, n, evk, Ychunk + (size_t)oA * 2 * n * N, p.in_ntt != 0, b1, C1,
                                     yo + (size_t)oA * 2 * (n - 1) * N, split, nullptr, ktB));
                if (cudaEventRecord(split_ev[1], split) != cudaSuccess ||
                    cudaStreamWaitEvent(st, split_ev[1], 0) != cudaSuccess)
                    return fail(BCN_E_CUDA, "bcn_eval: join failed");
            }
        }
        x = y;
    }
    const bcn_layer_plan &pl = m->layers.back();
    if (pl.in_ntt || pl.square) {  // back to coefficient form
        const int lout = pl.square ? pl.level - 1 : pl.level;
        Timed tm(prof, st, BCN_KERNEL_SQUARE, 2.0 * pl.n_out * 2 * lout * (double)N * 4);
        BCN_TRY(launch_ntt(c, out, (size_t)pl.n_out * 2 * lout, data_map(lout), true, st));
    }
    return BCN_OK;
}

static size_t pts_words(const bcn_model *m, int a_idx) {
    int a = 0;
    for (auto &p : m->layers)
        if (p.add) {
            if (a == a_idx) return (size_t)p.n_out * p.level * m->ctx->N;
            a++;
        }
    return 0;
}

bcn_status bcn_eval_host_workspace_bytes(const bcn_model *m, size_t *bytes) {
    if (!m || !bytes) return fail(BCN_E_INVAL, "bcn_eval_host_workspace_bytes: null argument");
    size_t b = 0;
    bcn_eval_workspace_bytes(m, &b);
    const bcn_ctx *c = m->ctx;
    b = align_up(b);
    b += align_up((size_t)m->layers.front().n_in * 2 * c->L * c->N * 4);
    int n_add = 0;
    for (auto &p : m->layers) n_add += p.add;
    for (int a = 0; a < n_add; a++) b += align_up(pts_words(m, a) * 4);
    b += align_up((size_t)m->layers.back().n_out * 2 * m->out_level * c->N * 4);
    *bytes = b;
    return BCN_OK;
}

bcn_status bcn_eval_host(const bcn_model *m, const uint32_t *evk, const uint32_t *cts_h,
                         const uint32_t *const *pts_h, uint32_t *out_h, void *ws, size_t ws_bytes, void *stream) {
    BCN_TRY(bcn_eval_host_async(m, evk, cts_h, pts_h, out_h, ws, ws_bytes, stream));
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return fail(BCN_E_CUDA, std::string("bcn_eval_host: ") + cudaGetErrorString(e));
    return BCN_OK;
}

// with `seeded`, cts_h holds c0 alone ([n_in][L][N]) and c1 is drawn on the
// device from the seed
static bcn_status eval_host_async_impl(const bcn_model *m, const uint32_t *evk, const uint32_t *cts_h,
                                       const uint32_t *const *pts_h, uint32_t *out_h, void *ws, size_t ws_bytes,
                                       void *stream, bool seeded, uint64_t seed,
                                       const int64_t *const *feats_i64 = nullptr);

bcn_status bcn_eval_host_async(const bcn_model *m, const uint32_t *evk, const uint32_t *cts_h,
                               const uint32_t *const *pts_h, uint32_t *out_h, void *ws, size_t ws_bytes,
                               void *stream) {
    return eval_host_async_impl(m, evk, cts_h, pts_h, out_h, ws, ws_bytes, stream, false, 0);
}

bcn_status bcn_eval_host_seeded_async(const bcn_model *m, const uint32_t *evk, const uint32_t *c0_h, uint64_t seed,
                                      const uint32_t *const *pts_h, uint32_t *out_h, void *ws, size_t ws_bytes,
                                      void *stream) {
    return eval_host_async_impl(m, evk, c0_h, pts_h, out_h, ws, ws_bytes, stream, true, seed);
}

bcn_status bcn_eval_host_compact_async(const bcn_model *m, const uint32_t *evk, const uint32_t *c0_h, uint64_t seed,
                                       const int64_t *const *feats_h, uint32_t *out_h, void *ws, size_t ws_bytes,
                                       void *stream) {
    if (!feats_h) return fail(BCN_E_INVAL, "bcn_eval_host_compact_async: null feature list");
    return eval_host_async_impl(m, evk, c0_h, nullptr, out_h, ws, ws_bytes, stream, true, seed, feats_h);
}

static bcn_status eval_host_async_impl(const bcn_model *m, const uint32_t *evk, const uint32_t *cts_h,
                                       const uint32_t *const *pts_h, uint32_t *out_h, void *ws, size_t ws_bytes,
                                       void *stream, bool seeded, uint64_t seed, const int64_t *const *feats_i64) {
    if (!m || !cts_h || !out_h) return fail(BCN_E_INVAL, "bcn_eval_host: null argument");
    if (seeded && m->stack != 1) return fail(BCN_E_INVAL, "bcn_eval_host_seeded_async: single-request models only");
    const bcn_ctx *c = m->ctx;
    BCN_TRY(check_device(c));
    size_t need = 0, eval_need = 0;
    bcn_eval_host_workspace_bytes(m, &need);
    bcn_eval_workspace_bytes(m, &eval_need);
    if (ws_bytes < need || !ws) return fail(BCN_E_BUDGET, "bcn_eval_host: workspace too small");
    int n_add = 0;
    for (auto &l : m->layers) n_add += l.add;
    for (int a = 0; a < n_add; a++)
        if (feats_i64 ? !feats_i64[a] : (!pts_h || !pts_h[a]))
            return fail(BCN_E_INVAL, "bcn_eval_host: missing feature plaintexts");
    cudaStream_t st = (cudaStream_t)stream;
    // Host-to-device copies go out in kCopyLanes parts on as many streams (the
    // copies run side by side), each after the caller's earlier work on `st`
    // (the workspace may still be in use); layer l waits only for its inputs,
    // so the later layers' features copy while the first layers compute.
    constexpr int kCopyLanes = 4;
    bcn_model *mm = const_cast<bcn_model *>(m);
    std::lock_guard<std::mutex> lock(mm->copy_mu);
    if (mm->copy_streams.empty()) {
        for (int i = 0; i < kCopyLanes; i++) {
            cudaStream_t s2 = nullptr;
            if (cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking) != cudaSuccess)
                return fail(BCN_E_CUDA, "bcn_eval_host: stream creation failed");
            mm->copy_streams.push_back(s2);
        }
    }
    std::vector<cudaEvent_t> events;
    auto new_event = [&](cudaEvent_t *e) {
        if (cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess) return false;
        events.push_back(*e);
        return true;
    };
    auto cleanup = [&](bcn_status s, const char *msg) {
        for (cudaEvent_t e : events) cudaEventDestroy(e);
        return s == BCN_OK ? BCN_OK : fail(s, msg);
    };
    // The copies overwrite the workspace's staging area: they wait for the last
    // evaluation that read it (its event), or, the first time a workspace is
    // seen, for everything queued on `st` so far.
    cudaEvent_t start;
    auto it = mm->staging_free.find(ws);
    if (it != mm->staging_free.end()) {
        start = it->second;
    } else if (!new_event(&start) || cudaEventRecord(start, st) != cudaSuccess) {
        return cleanup(BCN_E_CUDA, "bcn_eval_host: event failed");
    }
    for (cudaStream_t s2 : mm->copy_streams)
        if (cudaStreamWaitEvent(s2, start, 0) != cudaSuccess) return cleanup(BCN_E_CUDA, "bcn_eval_host: event wait");
    // one buffer: kCopyLanes parts, one event per part
    auto copy_in = [&](void *dst, const void *src, size_t bytes, std::vector<cudaEvent_t> &ready) {
        const size_t part = (bytes / kCopyLanes + 255) / 256 * 256;
        for (int i = 0; i < kCopyLanes; i++) {
            const size_t off = (size_t)i * part;
            if (off >= bytes) break;
            const size_t nb = std::min(part, bytes - off);
            cudaEvent_t e;
            if (cudaMemcpyAsync((char *)dst + off, (const char *)src + off, nb, cudaMemcpyHostToDevice,
                                mm->copy_streams[i]) != cudaSuccess ||
                !new_event(&e) || cudaEventRecord(e, mm->copy_streams[i]) != cudaSuccess)
                return false;
            ready.push_back(e);
        }
        return true;
    };
    char *p = reinterpret_cast<char *>(ws) + align_up(eval_need);
    const size_t cts_b = (size_t)m->layers.front().n_in * 2 * c->L * c->N * 4;
    uint32_t *cts_d = reinterpret_cast<uint32_t *>(p);
    p += align_up(cts_b);
    std::vector<std::vector<cudaEvent_t>> ready(m->layers.size());
    if (!seeded) {
        if (!copy_in(cts_d, cts_h, cts_b, ready[0])) return cleanup(BCN_E_CUDA, "bcn_eval_host: input copy failed");
    } else {
        // c0 rows into their ciphertexts' first halves, then c1 drawn in place,
        // kCopyLanes ranges of ciphertexts side by side
        const int n_in = m->layers.front().n_in;
        const size_t poly = (size_t)c->L * c->N;
        const int per = (n_in + kCopyLanes - 1) / kCopyLanes;
        for (int k = 0; k < kCopyLanes; k++) {
            const int lo = k * per, hi = std::min(n_in, lo + per);
            if (lo >= hi) break;
            cudaStream_t cs = mm->copy_streams[k];
            if (cudaMemcpy2DAsync(cts_d + (size_t)lo * 2 * poly, 2 * poly * 4, cts_h + (size_t)lo * poly, poly * 4,
                                  poly * 4, (size_t)(hi - lo), cudaMemcpyHostToDevice, cs) != cudaSuccess)
                return cleanup(BCN_E_CUDA, "bcn_eval_host: input copy failed");
            const bcn_status es = launch_expand_c1(c, cts_d + (size_t)lo * 2 * poly, hi - lo, c->L, seed, lo, cs);
            if (es != BCN_OK) return cleanup(es, bcn_last_error());
            cudaEvent_t e;
            if (!new_event(&e) || cudaEventRecord(e, cs) != cudaSuccess)
                return cleanup(BCN_E_CUDA, "bcn_eval_host: event failed");
            ready[0].push_back(e);
        }
    }
    std::vector<const uint32_t *> pts_d;
    // integer features: copied into the evaluation scratch's first ciphertext
    // buffer (idle until this evaluation's first layer writes it), reduced mod
    // each prime into the staging area on the copy streams; the first layer
    // waits for all of them, the layer of each (and its feature transform) for
    // its own
    char *i64 = reinterpret_cast<char *>(ws);
    size_t i64_used = 0;
    for (size_t l = 0, a = 0; l < m->layers.size(); l++) {
        if (!m->layers[l].add) continue;
        const size_t b = pts_words(m, (int)a) * 4;
        if (!feats_i64) {
            if (!copy_in(p, pts_h[a], b, ready[l])) return cleanup(BCN_E_CUDA, "bcn_eval_host: feature copy failed");
        } else {
            const bcn_layer_plan &lp = m->layers[l];
            const size_t row = (size_t)c->N * 8, rows_b = (size_t)lp.n_out * row;
            if (i64_used + rows_b > m->ws_x_bytes)
                return cleanup(BCN_E_BUDGET, "bcn_eval_host_compact_async: the integer features exceed the scratch");
            int64_t *src_d = reinterpret_cast<int64_t *>(i64 + i64_used);
            i64_used += align_up(rows_b);
            const int per = (lp.n_out + kCopyLanes - 1) / kCopyLanes;
            for (int k = 0; k < kCopyLanes; k++) {
                const int lo = k * per, hi = std::min(lp.n_out, lo + per);
                if (lo >= hi) break;
                cudaStream_t cs = mm->copy_streams[k];
                if (cudaMemcpyAsync(src_d + (size_t)lo * c->N, feats_i64[a] + (size_t)lo * c->N,
                                    (size_t)(hi - lo) * row, cudaMemcpyHostToDevice, cs) != cudaSuccess)
                    return cleanup(BCN_E_CUDA, "bcn_eval_host: feature copy failed");
                for (int v0 = lo; v0 < hi; v0 += 65535) {
                    const int nv = std::min(65535, hi - v0);
                    const bcn_status es = launch_expand_i64(c, src_d + (size_t)v0 * c->N, nv, lp.level,
                                                            reinterpret_cast<uint32_t *>(p) + (size_t)v0 * lp.level * c->N,
                                                            cs);
                    if (es != BCN_OK) return cleanup(es, bcn_last_error());
                }
                cudaEvent_t e;
                if (!new_event(&e) || cudaEventRecord(e, cs) != cudaSuccess)
                    return cleanup(BCN_E_CUDA, "bcn_eval_host: event failed");
                ready[0].push_back(e);
                if (l != 0) ready[l].push_back(e);
            }
        }
        pts_d.push_back(reinterpret_cast<const uint32_t *>(p));
        p += align_up(b);
        a++;
    }
    uint32_t *out_d = reinterpret_cast<uint32_t *>(p);
    bcn_status s = eval_impl(m, evk, cts_d, pts_d.data(), out_d, ws, eval_need, stream, &ready);
    if (s != BCN_OK) return cleanup(s, bcn_last_error());
    {  // the staging area is free again once this evaluation has run
        cudaEvent_t done;
        if (cudaEventCreateWithFlags(&done, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventRecord(done, st) != cudaSuccess)
            return cleanup(BCN_E_CUDA, "bcn_eval_host: event failed");
        auto old_it = mm->staging_free.find(ws);
        if (old_it != mm->staging_free.end()) cudaEventDestroy(old_it->second);
        mm->staging_free[ws] = done;
    }
    const size_t out_b = (size_t)m->layers.back().n_out * 2 * m->out_level * c->N * 4;
    if (cudaMemcpyAsync(out_h, out_d, out_b, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return cleanup(BCN_E_CUDA, "bcn_eval_host: output copy failed");
    return cleanup(BCN_OK, "");  // events are released once the device has passed them
}

// ------------------------------------------------------------- kernel timing
bcn_status bcn_profile_enable(bcn_model *m, int enable) {
    if (!m) return fail(BCN_E_INVAL, "bcn_profile_enable: null model");
    Profiler &p = m->prof;
    if (!p.recs.empty()) cudaDeviceSynchronize();
    p.on = enable != 0;
    p.recs.clear();
    p.used = 0;
    for (int k = 0; k < BCN_KERNEL_COUNT; k++) { p.ms[k] = 0; p.launches[k] = 0; p.bytes[k] = 0; }
    return BCN_OK;
}

bcn_status bcn_profile_read(bcn_model *m, int cls, double *ms, long long *launches, double *bytes) {
    if (!m || cls < 0 || cls >= BCN_KERNEL_COUNT) return fail(BCN_E_INVAL, "bcn_profile_read: bad argument");
    Profiler &p = m->prof;
    for (const auto &r : p.recs) {
        if (cudaEventSynchronize(p.ev[r.e1]) != cudaSuccess) return fail(BCN_E_CUDA, "bcn_profile_read: event wait");
        float t = 0;
        cudaEventElapsedTime(&t, p.ev[r.e0], p.ev[r.e1]);
        p.ms[r.cls] += t;
        p.launches[r.cls] += r.kernels;
        p.bytes[r.cls] += r.bytes;
    }
    p.recs.clear();
    p.used = 0;
    if (ms) *ms = p.ms[cls];
    if (launches) *launches = p.launches[cls];
    if (bytes) *bytes = p.bytes[cls];
    return BCN_OK;
}

// --------------------------------------------------------- single operations
bcn_status bcn_op_ntt(const bcn_ctx *c, uint32_t *data, int n_poly, int level, int inverse, void *stream) {
    BCN_TRY(check_device(c));
    if (!data || !aligned16(data) || n_poly < 0 || level < 1 || level > c->L)
        return fail(BCN_E_INVAL, "bcn_op_ntt: bad argument");
    return launch_ntt(c, data, (size_t)n_poly * level, data_map(level), inverse != 0, (cudaStream_t)stream);
}

bcn_status bcn_op_mac(const bcn_ctx *c, int level, int n_in, int n_out, int K, const int32_t *idx, const int8_t *w,
                      const uint32_t *in, const uint32_t *pt, uint32_t *out, void *stream) {
    BCN_TRY(check_device(c));
    if (!idx || !w || !in || !out || level < 1 || level > c->L || n_in < 0 || n_out < 0 || K < 0 ||
        K > kMaxMacTaps)
        return fail(BCN_E_INVAL, "bcn_op_mac: bad argument");
    if (!aligned16(in) || !aligned16(out) || (pt && !aligned16(pt)))
        return fail(BCN_E_INVAL, "bcn_op_mac: buffers must be 16-byte aligned");
    {  // every tap must name an input ciphertext or be a zero tap
        std::vector<int32_t> h((size_t)n_out * K);
        if (!h.empty() && cudaMemcpy(h.data(), idx, h.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
            return fail(BCN_E_CUDA, "bcn_op_mac: reading idx failed");
        for (int32_t v : h)
            if (v < -1 || v >= n_in) return fail(BCN_E_INVAL, "bcn_op_mac: idx entry outside [-1, n_in)");
    }
    if (debug_on(c, (cudaStream_t)stream)) {
        BCN_TRY(debug_residues(c, in, 2 * (size_t)n_in, level, (cudaStream_t)stream));
        BCN_TRY(debug_residues(c, pt, (size_t)n_out, level, (cudaStream_t)stream));
        BCN_TRY(debug_outcome(c, (cudaStream_t)stream, "bcn_op_mac"));
    }
    // every output is a group of one with its own taps
    return launch_mac(c, level, K, n_out, 1, idx, w, nullptr, in, pt, out, (cudaStream_t)stream);
}

bcn_status bcn_op_workspace_bytes(const bcn_ctx *c, int level, int n_ct, size_t *bytes) {
    if (!c || !bytes || level < 1 || level > c->L || n_ct < 0) return fail(BCN_E_INVAL, "bcn_op_workspace_bytes");
    *bytes = chunk_bytes(c, level, default_chunk(c, level, n_ct));
    return BCN_OK;
}

bcn_status bcn_op_tensor_square(const bcn_ctx *c, int level, const uint32_t *in, int n_ct, uint32_t *out, void *ws,
                                size_t ws_bytes, void *stream) {
    BCN_TRY(check_device(c));
    if (!in || !out || !aligned16(in) || !aligned16(out) || n_ct < 0 || level < 1 || level > c->L)
        return fail(BCN_E_INVAL, "bcn_op_tensor_square: bad argument");
    (void)ws;
    (void)ws_bytes;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t N = c->N;
    const CoreFns *f = core_fns(c);
    if (!f) return fail(BCN_E_INVAL, "unsupported ring degree");
    for (int o0 = 0; o0 < n_ct; o0 += 32768) {
        const int C = std::min(32768, n_ct - o0);
        uint32_t *o = out + (size_t)o0 * 3 * level * N;
        BCN_TRY(f->square(c, level, in + (size_t)o0 * 2 * level * N, o, nullptr, C, false, st));
        // d0 and d1 leave the kernel in the NTT domain
        BCN_TRY(launch_ntt_strided(c, o, 2 * (size_t)level, C, 3 * (size_t)level * N, data_map(level), true, st));
    }
    return BCN_OK;
}

bcn_status bcn_op_square_relin_rescale(const bcn_ctx *c, int level, const uint32_t *evk, const uint32_t *in,
                                       int n_ct, uint32_t *out, void *ws, size_t ws_bytes, void *stream) {
    BCN_TRY(check_device(c));
    if (level < 2 || level > c->L) return fail(BCN_E_LEVEL, "bcn_op_square_relin_rescale: level must be >= 2");
    size_t need = 0;
    BCN_TRY(bcn_op_workspace_bytes(c, level, n_ct, &need));
    if (ws_bytes < need || !ws) return fail(BCN_E_BUDGET, "bcn_op_square_relin_rescale: workspace too small");
    if (!in || !out || !evk || !aligned16(in) || !aligned16(out) || !aligned16(evk))
        return fail(BCN_E_INVAL, "bcn_op_square_relin_rescale: buffers");
    cudaStream_t st = (cudaStream_t)stream;
    BCN_TRY(debug_check_input(c, in, 2 * (size_t)n_ct, level, st, "bcn_op_square_relin_rescale"));
    const int n = level, chunk = default_chunk(c, level, n_ct);
    const size_t N = c->N;
    ChunkBufs b = carve_chunk(c, n, chunk, reinterpret_cast<char *>(ws));
    for (int o0 = 0; o0 < n_ct; o0 += chunk) {
        const int C = std::min(chunk, n_ct - o0);
        uint32_t *o = out + (size_t)o0 * 2 * (n - 1) * N;
        BCN_TRY(square_chunk(c, n, evk, in + (size_t)o0 * 2 * n * N, false, b, C, o, st));
        BCN_TRY(launch_ntt(c, o, (size_t)C * 2 * (n - 1), data_map(n - 1), true, st));
    }
    return BCN_OK;
}

bcn_status bcn_op_mul_plain_rescale(const bcn_ctx *c, int level, const uint32_t *in, int n_ct, const uint32_t *pt,
                                    uint32_t *out, void *ws, size_t ws_bytes, void *stream) {
    BCN_TRY(check_device(c));
    if (level < 2 || level > c->L) return fail(BCN_E_LEVEL, "bcn_op_mul_plain_rescale: level must be >= 2");
    if (n_ct < 0) return fail(BCN_E_INVAL, "bcn_op_mul_plain_rescale: bad count");
    if (n_ct == 0) return BCN_OK;
    size_t need = 0;
    BCN_TRY(bcn_op_workspace_bytes(c, level, n_ct, &need));
    if (!ws || ws_bytes < need) return fail(BCN_E_BUDGET, "bcn_op_mul_plain_rescale: workspace too small");
    if (!in || !out || !pt || !aligned16(in) || !aligned16(out) || !aligned16(pt) || !aligned16(ws))
        return fail(BCN_E_INVAL, "bcn_op_mul_plain_rescale: null or unaligned buffer");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t N = c->N, ct_words = 2 * (size_t)level * N;
    const size_t u_bytes = align_up((size_t)level * N * 4);
    uint32_t *U = reinterpret_cast<uint32_t *>(ws);
    uint32_t *X = reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(ws) + u_bytes);
    const size_t fit = (ws_bytes - u_bytes) / (ct_words * 4);
    const int chunk = (int)std::min<size_t>({fit, (size_t)n_ct, (size_t)(65535 / (2 * level))});
    if (chunk < 1) return fail(BCN_E_BUDGET, "bcn_op_mul_plain_rescale: workspace too small");
    if (cudaMemcpyAsync(U, pt, (size_t)level * N * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return fail(BCN_E_CUDA, "bcn_op_mul_plain_rescale: copy failed");
    BCN_TRY(launch_ntt(c, U, (size_t)level, data_map(level), false, st));
    for (int o0 = 0; o0 < n_ct; o0 += chunk) {
        const int C = std::min(chunk, n_ct - o0);
        if (cudaMemcpyAsync(X, in + (size_t)o0 * ct_words, (size_t)C * ct_words * 4, cudaMemcpyDeviceToDevice, st) !=
            cudaSuccess)
            return fail(BCN_E_CUDA, "bcn_op_mul_plain_rescale: copy failed");
        const size_t rows = (size_t)2 * level * C;
        BCN_TRY(launch_ntt(c, X, rows, data_map(level), false, st));
        k_mul_ntt<<<dim3((unsigned)((N + 255) / 256), (unsigned)rows), 256, 0, st>>>(X, U, level, (int)N, c->d_pc);
        BCN_TRY(check_launch("k_mul_ntt"));
        BCN_TRY(launch_ntt(c, X, rows, data_map(level), true, st));
        k_rescale<<<dim3((unsigned)((N + 255) / 256), 2, C), 256, 0, st>>>(
            X, out + (size_t)o0 * 2 * (level - 1) * N, level, (int)N, ks_dev(c), c->d_pc);
        BCN_TRY(check_launch("k_rescale"));
    }
    return BCN_OK;
}

bcn_status bcn_op_rescale(const bcn_ctx *c, int level, const uint32_t *in, int n_ct, uint32_t *out, void *stream) {
    BCN_TRY(check_device(c));
    if (level < 2 || level > c->L) return fail(BCN_E_LEVEL, "bcn_op_rescale: level must be >= 2");
    if (!in || !out || n_ct < 0) return fail(BCN_E_INVAL, "bcn_op_rescale: bad argument");
    const size_t N = c->N;
    for (int z0 = 0; z0 < n_ct; z0 += 65535) {  // grid.z limit
        const int nz = std::min(65535, n_ct - z0);
        k_rescale<<<dim3((c->N + 255) / 256, 2, nz), 256, 0, (cudaStream_t)stream>>>(
            in + (size_t)z0 * 2 * level * N, out + (size_t)z0 * 2 * (level - 1) * N, level, c->N, ks_dev(c), c->d_pc);
        BCN_TRY(check_launch("k_rescale"));
    }
    return BCN_OK;
}

}  // extern "C"
