// Integer-weight MAC on the fifth-generation tensor cores (tcgen05).
//
// The MAC of a layer group is a dense contraction
//     out[o][col] = sum_t w[o][t] * x[t][col]   (exact, then mod q),
// int8 weights times residues below 2^30 (Sec. 3.2: the ciphertext branch's
// linear layers use integer weights, so a MAC is plain integer arithmetic on
// the residues).  The tensor cores have no exact wide-integer path here, so a
// residue is split into its 4 bytes and each byte plane is one fp16 GEMM: a
// byte v sits in a half as the subnormal v * 2^-24 (the half's bit pattern is
// the byte itself, so a byte permute and a mask make two taps' halves),
// weights (-127..127) are exact, their products are exact multiples of 2^-24,
// and every partial sum of at most 512 taps stays below 512 * 255 * 127 < 2^24
// of those units, so the fp32 accumulation in tensor memory is exact.  The
// epilogue scales by 2^24, recombines the planes in int64
// (sum_b plane_b * 2^{8b}), adds a multiple of q that makes the sum
// non-negative and reduces mod q (Barrett), then adds the feature plaintext.
//
// One CTA: 128 coefficient columns (the MMA's M, one tensor-memory lane
// each) x one tile of at most 64 outputs (N, padded to a multiple of 16) of
// one group, all taps.  The weights of the tile are staged once in shared
// memory (B, K-major); the residues of a slab of 16 or 32 taps at a time (16
// for tiles of at most 32 outputs, whose CTAs fit 4 to an SM) arrive by
// cp.async in a ring of 3 stages (two slabs load while one converts) and are
// split into the 4 fp16 planes of A (K-major) by the two threads that own the
// column.
// One elected thread issues the MMAs and commits them to an mbarrier; the
// wait on it is bounded and records a status word on timeout.  Operand layout
// is the no-swizzle canonical K-major form: 8 rows x 16 bytes per core matrix,
// core matrices 128 bytes apart along K (LBO) and one row group apart along
// M/N (SBO).
#include <algorithm>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "device_api.h"
#include "device_math.cuh"

namespace bcn {

namespace {

constexpr int kRows = 128;                       // columns per CTA (MMA M)
constexpr int kThreads = 256;                    // two threads per column
constexpr int kABuf = 1;                         // A buffers (two measured slower: they halve the CTAs per SM)
constexpr int kPlanes = 4;                       // bytes of a residue
constexpr int kStages = 3;                       // raw slabs in shared memory

// Two shapes, chosen per layer by its output tile (mac_tc_plan):
//   tiles of at most 32 outputs: 16-tap slabs, registers for 4 CTAs per SM,
//     epilogue steps of 8 outputs (4 CTAs x 4 planes x 32 columns fill the
//     512 tensor-memory columns): the CIFAR-shaped conv2 layer 1.34 ms against
//     1.69 ms with the other shape;
//   wider tiles: 32-tap slabs, 2 CTAs per SM, epilogue steps of 16 outputs
//     (the CryptoNets-scale dense layer: 0.227 ms against 0.240 ms).
template <int SLAB>
struct TcSlab {
    static_assert(SLAB == 16 || SLAB == 32, "slabs of 16 or 32 taps");
    static constexpr int kStageBytes = SLAB * kRows * 4;   // raw residues of one slab
    static constexpr int kPlaneBytes = kRows * SLAB * 2;   // one fp16 plane of a slab
    static constexpr int kABytes = kPlanes * kPlaneBytes;  // one A buffer
    static constexpr uint32_t kSboA = (SLAB / 8) * 128;    // bytes between row groups of a plane
};
constexpr int kWaitLimit = 1 << 20;              // mbarrier polls before giving up

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start, LBO, SBO (bytes, 16-byte units),
// descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t mat_desc(uint32_t start, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((start >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// instruction descriptor, kind::f16: fp32 accumulator, fp16 A and B, both K-major
__host__ __device__ constexpr uint32_t instr_desc(int M, int N) {
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// two residues' byte b as a pair of subnormal halves (byte v is the half
// v * 2^-24): tap k in the low half, tap k + 1 in the high
__device__ __forceinline__ uint32_t byte_pair(uint32_t x0, uint32_t x1, int b) {
    const uint32_t sel = (uint32_t)b | ((uint32_t)b << 4) | ((uint32_t)(4 + b) << 8) | ((uint32_t)(4 + b) << 12);
    return __byte_perm(x0, x1, sel) & 0x00FF00FFu;
}

__device__ __forceinline__ void tmem_ld8(uint32_t addr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(addr));
}

__device__ __forceinline__ void tmem_ld16(uint32_t addr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(addr));
}

template <int E>
__device__ __forceinline__ void tmem_ld(uint32_t addr, uint32_t (&r)[E]) {
    if constexpr (E == 16)
        tmem_ld16(addr, r);
    else
        tmem_ld8(addr, r);
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    for (int i = 0; i < kWaitLimit; i++) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// 16-byte asynchronous copy global -> shared; zero-filled when !valid
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}

// residues of slab taps [t0, t0 + SLAB) of columns [col0, col0 + 128) into a
// stage ([tap][column] words), as one cp.async group
template <int SLAB>
__device__ __forceinline__ void stage_slab(uint32_t stage, const uint32_t *__restrict__ in, const int32_t *sidx,
                                           int t0, size_t cols, size_t col0, int tid) {
#pragma unroll
    for (int i = 0; i < TcSlab<SLAB>::kStageBytes / 16 / kThreads; i++) {
        const int c = tid + i * kThreads, tap = c >> 5, q4 = c & 31;
        const int s = sidx[t0 + tap];
        const uint32_t *src = s >= 0 ? in + (size_t)s * cols + col0 + 4 * q4 : in;
        cp_async16(stage + (uint32_t)(tap * kRows * 4 + q4 * 16), src, s >= 0);
    }
}

}  // namespace

// grid (n_groups * tiles, 2 level N / 128), 256 threads.  w16: per output tile
// the fp16 weights [NT][Kpad] in the canonical K-major layout (zero rows past
// the tile's outputs, zero columns past K).  Kpad is a multiple of kSlab.
// Shared memory: kStages raw stages (cp.async, kStages - 1 slabs in flight
// ahead of the one being converted), the fp16 planes of one slab (A), the
// tile's weights (B), the tap indices, the mbarrier.
template <int SLAB, int MINB, int EPI>
__global__ void __launch_bounds__(kThreads, MINB) k_mac_tc(const uint32_t *__restrict__ in, uint32_t *__restrict__ out,
                                                     const int32_t *__restrict__ gidx, const uint4 *__restrict__ w16,
                                                     const int32_t *__restrict__ gout,
                                                     const uint32_t *__restrict__ pt, int K, int Kpad, int n_go,
                                                     int tile_out, int NT, int t_lo, int n_tl, int level, int N,
                                                     int g_base, int store_natural, const PrimeConst *__restrict__ pc,
                                                     uint32_t tmem_cols, uint32_t *__restrict__ status) {
    constexpr int kSlab = SLAB, kStageBytes = TcSlab<SLAB>::kStageBytes, kPlaneBytes = TcSlab<SLAB>::kPlaneBytes;
    constexpr int kABytes = TcSlab<SLAB>::kABytes;
    constexpr uint32_t kSboA = TcSlab<SLAB>::kSboA;
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char *S = sm;                          // [kStages][kSlab][kRows] u32
    unsigned char *A = sm + kStages * kStageBytes;  // [kABuf][kPlanes] planes
    unsigned char *B = A + kABuf * kABytes;         // [NT][Kpad] fp16
    int32_t *sidx = reinterpret_cast<int32_t *>(B + (size_t)NT * Kpad * 2);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sidx + Kpad);  // [kABuf]: MMAs of the slabs in A buffer b
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + kABuf);
    volatile int *flag = reinterpret_cast<volatile int *>(tslot + 1);
    int32_t *sgo = reinterpret_cast<int32_t *>(tslot + 2);  // [NT] the tile's output indices

    const int tid = threadIdx.x, warp = tid >> 5, r = tid & (kRows - 1), half = tid >> 7;
    // output tiles vary fastest over the grid: the CTAs that run together read
    // the same columns of every input, which stay in L2 between them
    const int g = g_base + (int)blockIdx.x / n_tl, tile = t_lo + (int)blockIdx.x % n_tl;
    const int o0 = tile * tile_out, no = min(tile_out, n_go - o0);
    const size_t cols = (size_t)2 * level * N;
    const size_t col0 = (size_t)blockIdx.y * kRows, col = col0 + r;
    const int n_slabs = Kpad / kSlab;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)),
                     "r"(tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
#pragma unroll
        for (int b = 0; b < kABuf; b++) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(mbar + b)));
        asm volatile("fence.mbarrier_init.release.cluster;");
        *flag = 0;
    }
    for (int t = tid; t < Kpad; t += kThreads) sidx[t] = t < K ? gidx[(size_t)g * K + t] : -1;
    for (int o = tid; o < no; o += kThreads) sgo[o] = gout != nullptr ? gout[(size_t)g * n_go + o0 + o] : g * n_go + o0 + o;
    __syncthreads();  // sidx
    const uint32_t s_base = smem_addr(S);
#pragma unroll
    for (int k = 0; k < kStages - 1; k++) {  // the first slabs, one cp.async group each
        if (k < n_slabs) stage_slab<SLAB>(s_base + (uint32_t)(k * kStageBytes), in, sidx, k * kSlab, cols, col0, tid);
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    {
        const uint4 *src = w16 + (size_t)tile * ((size_t)NT * Kpad * 2 / 16);
        uint4 *dst = reinterpret_cast<uint4 *>(B);
        for (int i = tid; i < NT * Kpad * 2 / 16; i += kThreads) dst[i] = __ldg(src + i);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tslot;
    const uint32_t a_base0 = smem_addr(A), b_base = smem_addr(B), mb0 = smem_addr(mbar);
    const uint32_t idesc = instr_desc(kRows, NT);
    const uint32_t sbo_b = (uint32_t)(Kpad / 8) * 128;

    int sl = 0;  // after the loop: the slabs whose MMAs were issued and committed
    for (; sl < n_slabs; sl++) {
        // keep kStages - 1 slabs in flight: issue slab sl + kStages - 1 (its
        // stage was converted at iteration sl - 1), then wait for slab sl
        {
            const int nx = sl + kStages - 1;
            if (nx < n_slabs)
                stage_slab<SLAB>(s_base + (uint32_t)((nx % kStages) * kStageBytes), in, sidx, nx * kSlab, cols, col0,
                           tid);
            asm volatile("cp.async.commit_group;" ::: "memory");
            asm volatile("cp.async.wait_group %0;" ::"n"(kStages - 1) : "memory");
        }
        // A buffer ab held slab sl - kABuf: its MMAs (the (sl/kABuf - 1)-th
        // commit to mbar[ab]) must be done before it is overwritten
        const int ab = sl % kABuf;
        const uint32_t a_base = a_base0 + (uint32_t)(ab * kABytes), mb = mb0 + (uint32_t)(ab * 8);
        if (tid == 0 && sl >= kABuf && !mbar_wait(mb, (uint32_t)((sl / kABuf - 1) & 1))) *flag = 1;
        __syncthreads();  // slab sl is in its stage for every thread; A buffer ab is free
        if (*flag) break;
        {
            constexpr int TT = kSlab / 2;  // taps a thread converts
            const uint32_t *st = reinterpret_cast<const uint32_t *>(S + (sl % kStages) * kStageBytes);
            uint32_t x[TT];
#pragma unroll
            for (int j = 0; j < TT; j++) x[j] = st[(TT * half + j) * kRows + r];
#pragma unroll
            for (int h = 0; h < TT / 8; h++) {
                const int t8 = TT * half + 8 * h;
                const uint32_t off = (uint32_t)(r >> 3) * kSboA + (uint32_t)(t8 >> 3) * 128 + (r & 7) * 16;
#pragma unroll
                for (int b = 0; b < kPlanes; b++) {
                    uint4 v;
                    v.x = byte_pair(x[8 * h + 0], x[8 * h + 1], b);
                    v.y = byte_pair(x[8 * h + 2], x[8 * h + 3], b);
                    v.z = byte_pair(x[8 * h + 4], x[8 * h + 5], b);
                    v.w = byte_pair(x[8 * h + 6], x[8 * h + 7], b);
                    *reinterpret_cast<uint4 *>(A + ab * kABytes + b * kPlaneBytes + off) = v;
                }
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
            for (int b = 0; b < kPlanes; b++) {
#pragma unroll
                for (int j = 0; j < kSlab / 16; j++) {
                    const uint64_t ad = mat_desc(a_base + b * kPlaneBytes + j * 256, 128, kSboA);
                    const uint64_t bd = mat_desc(b_base + (uint32_t)(sl * (kSlab / 16) + j) * 256, 128, sbo_b);
                    const uint32_t d = tmem + (uint32_t)(b * NT);
                    const uint32_t acc = (sl > 0 || j > 0) ? 1u : 0u;
                    asm volatile(
                        "{\n\t.reg .pred p;\n\t"
                        "setp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
                        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb));
        }
    }
    // The last commit tracks every MMA issued before it.  On the normal path
    // this is the wait for the whole contraction.  After a timed-out wait (the
    // loop stopped before committing slab sl) it drains the MMAs still in
    // flight, again bounded, so that neither shared memory nor tensor memory
    // is released while they may read or write it; only if that wait gives up
    // too does the CTA go on to free its tensor memory regardless (there is no
    // unbounded way left that keeps the GPU answering).
    if (tid == 0 && sl > 0) {
        const int last = sl - 1;
        if (!mbar_wait(mb0 + (uint32_t)((last % kABuf) * 8), (uint32_t)((last / kABuf) & 1))) *flag = 1;
    }
    __syncthreads();
    asm volatile("cp.async.wait_group 0;" ::: "memory");

    if (*flag == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        // warp w reads tensor-memory lanes 32 (w mod 4) ..; the two warp halves
        // take alternate blocks of E outputs
        const uint32_t lanes = tmem + ((uint32_t)((warp & 3) * 32) << 16);
        const int i = (int)((col / N) % level), poly = (int)(col / ((size_t)level * N));
        const uint32_t q = pc[i].q;
        const uint64_t mu = pc[i].barrett;
        const long long offs = (long long)pc[i].mac_offset;
        constexpr int E = EPI;
        for (int ob = E * half; ob < NT; ob += 2 * E) {
            uint32_t f[kPlanes][E];
#pragma unroll
            for (int b = 0; b < kPlanes; b++) tmem_ld<E>(lanes + (uint32_t)(b * NT + ob), f[b]);
            const int nv = min(E, no - ob);  // live outputs of this block of E (may be <= 0)
            // the feature words of all E outputs are requested before any is used
            uint32_t pv[E];
#pragma unroll
            for (int o = 0; o < E; o++)
                pv[o] = pt != nullptr && poly == 0 && o < nv ? __ldg(pt + (size_t)sgo[ob + o] * level * N + col) : 0u;
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int o = 0; o < E; o++) {
                if (o < nv) {
                    long long v = offs;
#pragma unroll
                    for (int b = 0; b < kPlanes; b++)
                        v += (long long)__float2int_rn(__uint_as_float(f[b][o]) * 16777216.0f) << (8 * b);
                    // offs >= 2^58 and |sum| < 2^48: v is positive and below 2^59
                    const uint32_t res = add_mod(reduce59((uint64_t)v, q, mu), pv[o], q);
                    const int os = store_natural ? sgo[ob + o] : (g - g_base) * n_go + o0 + ob + o;
                    out[(size_t)os * cols + col] = res;
                }
            }
        }
    } else if (tid == 0) {
        atomicOr(status, 1u);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols));
    }
}

// ------------------------------------------------------------------ host side
static uint16_t half_of_int(int v) {  // exact for |v| < 2048
    if (v == 0) return 0;
    const uint16_t s = v < 0 ? 0x8000 : 0;
    int a = v < 0 ? -v : v, e = 0;
    while ((a >> (e + 1)) != 0) e++;
    const uint16_t mant = (uint16_t)(((uint32_t)a << (10 - e)) & 0x3FF);
    return (uint16_t)(s | ((e + 15) << 10) | mant);
}

bool mac_tc_eligible(const bcn_ctx *c, int K, int n_go) {
    const bool wide = n_go >= kMacTcMinOutputs || (n_go >= kMacTcMinOutputsLong && K >= kMacTcLongTaps);
    return K >= 1 && K <= kMacTcMaxTaps && wide && c->N >= kRows && c->N % kRows == 0;
}

template <int SLAB>
size_t mac_tc_smem_t(int NT, int Kpad) {
    using TS = TcSlab<SLAB>;
    return (size_t)kStages * TS::kStageBytes + (size_t)kABuf * TS::kABytes + (size_t)NT * Kpad * 2 +
           (size_t)Kpad * 4 + 8 * kABuf + 8 + (size_t)NT * 4 + 1024;
}
size_t mac_tc_smem(int NT, int Kpad, int slab) {
    return slab == 16 ? mac_tc_smem_t<16>(NT, Kpad) : mac_tc_smem_t<32>(NT, Kpad);
}

// the two kernel shapes (see TcSlab)
#define BCN_TC_NARROW k_mac_tc<16, 4, 8>
#define BCN_TC_WIDE k_mac_tc<32, 2, 16>

bcn_status mac_tc_plan(const bcn_ctx *c, int K, int n_go, const int8_t *w, MacTcPlan *p) {
    const int tiles = (n_go + 63) / 64;
    const int tile_out = (n_go + tiles - 1) / tiles;
    const int NT0 = (tile_out + 15) / 16 * 16;
    const int slab = NT0 <= 32 ? 16 : 32;
    const int NT = NT0, Kpad = (K + slab - 1) / slab * slab;
    uint32_t cols = 32;
    while (cols < (uint32_t)(kPlanes * NT)) cols *= 2;
    // weights per tile in the canonical K-major layout
    std::vector<uint16_t> h((size_t)tiles * NT * Kpad, 0);
    for (int tt = 0; tt < tiles; tt++) {
        const int o0 = tt * tile_out, no = std::min(tile_out, n_go - o0);
        uint16_t *dst = h.data() + (size_t)tt * NT * Kpad;
        for (int n = 0; n < no; n++)
            for (int k = 0; k < K; k++)
                dst[((size_t)(n / 8) * (Kpad / 8) + k / 8) * 64 + (n % 8) * 8 + (k % 8)] =
                    half_of_int(w[(size_t)(o0 + n) * K + k]);
    }
    if (cudaMalloc(&p->w16, h.size() * 2) != cudaSuccess) return fail(BCN_E_NOMEM, "MAC weight tables");
    if (cudaMemcpy(p->w16, h.data(), h.size() * 2, cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(BCN_E_CUDA, "upload of the MAC weight tables failed");
    // co-resident CTAs must fit the 512 tensor-memory columns of an SM: grow
    // the shared-memory request until they do
    size_t smem = mac_tc_smem(NT, Kpad, slab);
    for (;;) {
        int nb = 0;
        const void *kern = slab == 16 ? (const void *)BCN_TC_NARROW : (const void *)BCN_TC_WIDE;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kThreads, smem) != cudaSuccess)
            return fail(BCN_E_CUDA, "occupancy query for the tensor-core MAC failed");
        if (nb < 1) return fail(BCN_E_INVAL, "tensor-core MAC: shared memory does not fit");
        if ((uint32_t)nb * cols <= 512) break;
        smem += 4096;
    }
    p->tiles = tiles;
    p->tile_out = tile_out;
    p->NT = NT;
    p->Kpad = Kpad;
    p->tmem_cols = cols;
    p->smem = smem;
    p->slab = slab;
    return BCN_OK;
}

bcn_status mac_tc_setup() {
    if (cudaFuncSetAttribute(BCN_TC_NARROW, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024) != cudaSuccess ||
        cudaFuncSetAttribute(BCN_TC_WIDE, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024) != cudaSuccess)
        return fail(BCN_E_CUDA, "cudaFuncSetAttribute failed for the tensor-core MAC");
    return BCN_OK;
}

bcn_status launch_mac_tc(const bcn_ctx *c, const MacTcPlan &p, int level, int K, int n_groups, int n_go,
                         const int32_t *gidx, const int32_t *gout, const uint32_t *in, const uint32_t *pt,
                         uint32_t *out, cudaStream_t st, int g_base, bool store_natural, int t_lo, int n_tl) {
    const size_t cols = (size_t)2 * level * c->N;
    if (t_lo < 0 || n_tl < 1 || t_lo + n_tl > p.tiles) return fail(BCN_E_INVAL, "MAC tile range");
    if (cols / kRows > 65535) return fail(BCN_E_INVAL, "MAC: more than 65535 column blocks");
    dim3 grid((unsigned)(n_groups * n_tl), (unsigned)(cols / kRows));
    if (p.slab == 16)
        BCN_TC_NARROW<<<grid, kThreads, p.smem, st>>>(in, out, gidx, reinterpret_cast<const uint4 *>(p.w16), gout, pt,
                                                       K, p.Kpad, n_go, p.tile_out, p.NT, t_lo, n_tl, level, c->N,
                                                       g_base, store_natural ? 1 : 0, c->d_pc, p.tmem_cols,
                                                       c->d_status);
    else
        BCN_TC_WIDE<<<grid, kThreads, p.smem, st>>>(in, out, gidx, reinterpret_cast<const uint4 *>(p.w16), gout, pt,
                                                     K, p.Kpad, n_go, p.tile_out, p.NT, t_lo, n_tl, level, c->N,
                                                     g_base, store_natural ? 1 : 0, c->d_pc, p.tmem_cols,
                                                     c->d_status);
    return check_launch("k_mac_tc");
}

}  // namespace bcn
