// Host-side launch helpers shared by the device translation units.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "bcn_internal.h"

namespace bcn {

// Host-side NVTX range: names the library's phases (an evaluation, its layers,
// each kernel class's launches) on a profiler's timeline.  Header-only NVTX:
// with no tool attached a push or pop is a check of one function pointer.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// prime map of a buffer whose limbs cycle through the data primes q_0..q_{level-1}
inline PrimeMap data_map(int level) { return PrimeMap{level, level, 0}; }
// prime map of the extended basis Q_level u P: q_0..q_{level-1}, p_0..p_{K-1}
inline PrimeMap ext_map(const bcn_ctx *c, int level) { return PrimeMap{level + c->K, level, c->L - level}; }

__host__ __device__ inline int prime_of(const PrimeMap &m, int limb) {
    const int t = limb % m.period;
    return t < m.split ? t : t + m.offset;
}

// return the status of a call that fails
#define BCN_TRY(x)                          \
    do {                                    \
        bcn_status _s = (x);                \
        if (_s != BCN_OK) return _s;        \
    } while (0)

inline bcn_status check_launch(const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(BCN_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    return BCN_OK;
}

// basis-conversion tables as the kernels see them (layout: KsTables)
struct KsDev {
    const uint2 *dhat_inv, *dhat, *phat_inv, *phat, *pinv, *qtop_inv;
    const uint32_t *dprod, *pmod;
    int L, K, alpha, dnum_max, P;
};

inline KsDev ks_dev(const bcn_ctx *c) {
    const KsTables &t = c->ks;
    KsDev k;
    k.dhat_inv = reinterpret_cast<const uint2 *>(c->d_ks + t.off_dhat_inv);
    k.dhat = reinterpret_cast<const uint2 *>(c->d_ks + t.off_dhat);
    k.dprod = c->d_ks + t.off_dprod;
    k.phat_inv = reinterpret_cast<const uint2 *>(c->d_ks + t.off_phat_inv);
    k.phat = reinterpret_cast<const uint2 *>(c->d_ks + t.off_phat);
    k.pmod = c->d_ks + t.off_pmod;
    k.pinv = reinterpret_cast<const uint2 *>(c->d_ks + t.off_pinv);
    k.qtop_inv = reinterpret_cast<const uint2 *>(c->d_ks + t.off_qtop_inv);
    k.L = t.L; k.K = t.K; k.alpha = t.alpha; k.dnum_max = t.dnum_max; k.P = t.P;
    return k;
}

// Keys of a stacked evaluation (several requests of one model, each with its
// client's evaluation key): the ciphertexts of a square-layer chunk that starts
// at position ct_base of the layer's group-major order belong to request
// (ct_base + ct) / cts_per_key, and the chunk's key switch is launched once per
// request it covers, with that request's key.  n == 0: one key for the chunk.
constexpr int kMaxStack = 16;
struct KeyTable {
    const uint32_t *key[kMaxStack];
    int n, ct_base, cts_per_key;
};

// A batch of rotations for the hoisted key switch, passed by value: the
// prepared Galois key and the Galois element g of each (kRotBatch at most).
constexpr int kRotBatch = 32;
struct RotBatch {
    const uint32_t *gk[kRotBatch];
    uint32_t g[kRotBatch];
    uint32_t ginv[kRotBatch];
    int count;
};

// The NTT-based kernels of one ring degree (template instances live in
// cores_*.cu so they compile in parallel).
struct CoreFns {
    // in-place NTT of n_limbs limbs in each of n_groups groups `stride` words
    // apart; limb l uses prime prime_of(pm, l).  Forward: natural order ->
    // last-pass layout; inverse: back.
    bcn_status (*ntt)(const bcn_ctx *, uint32_t *data, size_t n_limbs, size_t n_groups, size_t stride, PrimeMap pm,
                      bool inverse, cudaStream_t);
    // Y [C][2][n][N] (coefficient form, or NTT domain when in_ntt) -> D [C][3][n][N]:
    // d0, d1 in the NTT domain, d2 in coefficient form; if D2N is not null, d2
    // in the NTT domain [C][n][N] too
    bcn_status (*square)(const bcn_ctx *, int n, const uint32_t *Y, uint32_t *D, uint32_t *D2N, int C, bool in_ntt,
                         cudaStream_t);
    // D (d2; D2N optional) -> ACC [C][2][n+K][N] (key-switching sums, coefficient
    // form; with ntt_out the data limbs in the NTT domain)
    bcn_status (*keyswitch)(const bcn_ctx *, int n, const uint32_t *D, const uint32_t *D2N, const uint32_t *evk,
                            uint32_t *acc, int C, bool ntt_out, cudaStream_t);
    // D (NTT-domain d0, d1) and ACC (the key switch's output with ntt_out) ->
    // OUT [C][2][n-1][N] (ModDown by P, add, rescale by q_{n-1}; NTT domain)
    bcn_status (*moddown_rescale)(const bcn_ctx *, int n, const uint32_t *D, const uint32_t *acc, uint32_t *out,
                                  int C, cudaStream_t);
    bcn_status (*setup)();
    // hoisted rotations: U [C][dnum][n+K][N] <- NTT-domain ModUp of every digit
    // of the ciphertexts' c1 (in [C][2][n][N], coefficient form)
    bcn_status (*modup_hoist)(const bcn_ctx *, int n, const uint32_t *in, uint32_t *U, int C, cudaStream_t);
    // ACC [C][rb.count][2][n+K][N] <- key switching of sigma_g(c1) for every
    // rotation of the batch (coefficient form, ready for ModDown)
    bcn_status (*ks_rot)(const bcn_ctx *, int n, const uint32_t *U, const RotBatch &rb, uint32_t *acc, int C,
                         cudaStream_t);
};
const CoreFns *core_fns(int logN, int alt = 0);  // nullptr if unsupported; alt: the alternative block shape
// the context's selected block shape (bcn_ctx_set_ntt_shape)
const CoreFns *core_fns(const bcn_ctx *c);
const CoreFns *core_fns_12_alt();
const CoreFns *core_fns_13_alt();
const CoreFns *core_fns_14_alt();
const CoreFns *core_fns_small(int logN);
const CoreFns *core_fns_12();
const CoreFns *core_fns_13();
const CoreFns *core_fns_14();

// square + relinearise + rescale of C ciphertexts Y [C][2][n][N] -> out [C][2][n-1][N],
// both in coefficient form, intermediates in d [C][3][n][N] and acc [C][2][n+K][N]
bcn_status square_relin_rescale_chunk(const bcn_ctx *c, int n, const uint32_t *evk, const uint32_t *Y, uint32_t *d,
                                      uint32_t *acc, int C, uint32_t *out, cudaStream_t st);

// in-place NTT of n_limbs limbs (limb l with prime prime_of(pm, l)); forward:
// natural order -> last-pass layout, inverse: back.  The strided form does it
// for n_groups groups `stride` words apart.
bcn_status launch_ntt(const bcn_ctx *c, uint32_t *data, size_t n_limbs, const PrimeMap &pm, bool inverse,
                      cudaStream_t st);
bcn_status launch_ntt_strided(const bcn_ctx *c, uint32_t *data, size_t n_limbs, size_t n_groups, size_t stride,
                              const PrimeMap &pm, bool inverse, cudaStream_t st);

// key-switching chunk of the op entry points (eval.cu): ciphertexts per chunk
// at level n for n_ct ciphertexts, and the chunk's buffers in a workspace of
// bcn_op_workspace_bytes: D [C][3][n][N], D2N [C][n][N], ACC [C][2][n+K][N]
int ks_default_chunk(const bcn_ctx *c, int n, int n_ct);
void ks_carve(const bcn_ctx *c, int n, int chunk, char *ws, uint32_t **d, uint32_t **d2n, uint32_t **acc);

// Tensor-core MAC (mac_tc.cu): used for groups of at most kMacTcMaxTaps taps
// (the fp32 sums stay exact) and at least kMacTcMinOutputs outputs, or at least
// kMacTcMinOutputsLong outputs when they have kMacTcLongTaps taps or more
// (measured: dense layers of 10 outputs and 80-100 taps are faster there, a
// 27-tap convolution with 16 outputs is not).
#ifndef BCN_TC_MIN_OUTPUTS
#define BCN_TC_MIN_OUTPUTS 32
#endif
constexpr int kMacTcMaxTaps = 512, kMacTcMinOutputs = BCN_TC_MIN_OUTPUTS;
constexpr int kMacTcMinOutputsLong = 10, kMacTcLongTaps = 64;
bool mac_tc_eligible(const bcn_ctx *c, int K, int n_go);
// w: [n_go][K] int8 weights shared by every group
bcn_status mac_tc_plan(const bcn_ctx *c, int K, int n_go, const int8_t *w, MacTcPlan *p);
bcn_status mac_tc_setup();
bcn_status launch_mac_tc(const bcn_ctx *c, const MacTcPlan &p, int level, int K, int n_groups, int n_go,
                         const int32_t *gidx, const int32_t *gout, const uint32_t *in, const uint32_t *pt,
                         uint32_t *out, cudaStream_t st, int g_base, bool store_natural, int t_lo, int n_tl);
bcn_status cores_setup_all();
// seeded ciphertexts: c1 of cts [n_ct][2][level][N] drawn from the seed (ciphertext
// ct takes the stream of index ct_base + ct); c0 untouched
bcn_status launch_expand_c1(const bcn_ctx *c, uint32_t *cts, int n_ct, int level, uint64_t seed, int ct_base,
                            cudaStream_t st);
// integer plaintexts: coeffs [n][N] (|m| < 2^63) -> pts [n][level][N], m mod q_i
bcn_status launch_expand_i64(const bcn_ctx *c, const int64_t *coeffs, int n, int level, uint32_t *pts,
                             cudaStream_t st);
// with the context's debug checks on (and the stream not capturing): every
// residue of polys [n_poly][level][N] below its prime, checked on the device,
// else BCN_E_INVAL naming `who`; a no-op otherwise
bcn_status debug_check_input(const bcn_ctx *c, const uint32_t *a, size_t n_poly, int level, cudaStream_t st,
                             const char *who);
// rescale of C coefficient-form ciphertexts: in [C][2][n][N] -> out [C][2][n-1][N]
bcn_status launch_rescale(const bcn_ctx *c, int n, const uint32_t *in, uint32_t *out, int C, cudaStream_t st);

}  // namespace bcn
