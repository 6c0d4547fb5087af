// Internal declarations shared by the host (.cpp) and device (.cu) sources of
// the library.  Not part of the public ABI (include/bcn.h is).
#pragma once

#include <cstdint>
#include <cstring>
#include <string>
#include <mutex>
#include <unordered_map>
#include <vector>

#include <cuda_runtime_api.h>
#include <vector_types.h>  // uint2

#include "bcn.h"

namespace bcn {

constexpr int kMaxPrimes = 28;  // L + K <= 24 + 4
constexpr int kMaxLogN = 14;

// error reporting -----------------------------------------------------------
void set_error(const std::string &msg);
bcn_status fail(bcn_status st, const std::string &msg);

// 64-bit helpers on the host --------------------------------------------------
inline uint64_t mulmod64(uint64_t a, uint64_t b, uint64_t m) {
    return (uint64_t)((unsigned __int128)a * b % m);
}
uint64_t powmod64(uint64_t a, uint64_t e, uint64_t m);
inline uint64_t invmod64(uint64_t a, uint64_t m) { return powmod64(a % m, m - 2, m); }  // m prime
inline uint32_t shoup_companion(uint32_t w, uint32_t q) { return (uint32_t)(((uint64_t)w << 32) / q); }

// per-prime constants, device resident ---------------------------------------
struct PrimeConst {
    uint32_t q;
    uint32_t qneg_inv;   // -q^{-1} mod 2^32 (Montgomery, R = 2^32)
    uint32_t r_mod;      // R mod q
    uint32_t r_shoup;    // Shoup companion of r_mod
    uint32_t ninv;       // N^{-1} mod q
    uint32_t ninv_shoup;
    uint32_t half;       // (q - 1) / 2: the largest residue whose centred value is >= 0
    uint32_t rn;         // R * N^{-1} mod q: Montgomery form of N^{-1}
    uint32_t rn_shoup;   // Shoup companion of rn
    uint32_t one;        // 1, read at run time: multiply-adds by it stay on the FMA pipe
    uint32_t nmod;       // N mod q (= N)
    uint32_t nmod_shoup; // Shoup companion of nmod
    uint64_t barrett;    // floor(2^64 / q)
    uint64_t mac_offset; // a multiple of q >= 2^58 (makes a signed MAC sum non-negative)
};

// which prime each limb of a batched buffer uses: t = limb % period, then
// prime index t if t < split, else t + offset
struct PrimeMap {
    int period, split, offset;
};

// basis-conversion constants, device resident (one blob) ----------------------
// ModUp at level n, digit j, prime i of the digit (local index u < alpha),
// target prime index P (0..L+K-1):
//   dhat_inv[n][j][u]     = (D_j / q_i)^{-1} mod q_i          (value, shoup)
//   dhat[n][j][u][P]      = (D_j / q_i) mod prime_P           (value, shoup)
//   dprod[n][j][P]        = D_j mod prime_P
// ModDown (target data prime i, special prime m):
//   phat_inv[m]           = (P / p_m)^{-1} mod p_m            (value, shoup)
//   phat[m][i]            = (P / p_m) mod q_i                 (value, shoup)
//   pmod[i]               = P mod q_i
//   pinv[i]               = P^{-1} mod q_i                    (value, shoup)
// Rescale dropping q_top (top = n - 1), target i < top:
//   qtop_inv[top][i]      = q_top^{-1} mod q_i                (value, shoup)
struct KsTables {
    int L, K, alpha, dnum_max, P;  // P = L + K
    // offsets (in uint32 words) into the device blob
    size_t off_dhat_inv, off_dhat, off_dprod, off_phat_inv, off_phat, off_pmod, off_pinv, off_qtop_inv;
    std::vector<uint32_t> host;   // the blob
    // index helpers (element = uint2 for (value, shoup) entries)
    size_t i_dhat_inv(int n, int j, int u) const { return ((size_t)(n * dnum_max + j) * alpha + u); }
    size_t i_dhat(int n, int j, int u, int p) const { return (((size_t)(n * dnum_max + j) * alpha + u) * P + p); }
    size_t i_dprod(int n, int j, int p) const { return ((size_t)(n * dnum_max + j) * P + p); }
};

}  // namespace bcn

// the opaque objects -------------------------------------------------------------
namespace bcn {
// Tensor-core MAC of a layer: fp16 weight tables per output tile and launch shape.
struct MacTcPlan {
    uint16_t *w16 = nullptr;  // [tiles][NT][Kpad] canonical K-major layout
    int tiles = 0, tile_out = 0, NT = 0, Kpad = 0;
    uint32_t tmem_cols = 0;
    size_t smem = 0;
    int slab = 32;  // taps per slab: 16 (tiles of at most 32 outputs) or 32
};
}  // namespace bcn

struct bcn_ctx {
    bcn_params params;
    int N, logN, L, K, alpha, dnum;
    int device;  // -1: host only
    int ntt_alt = 0;  // block shape of the NTT-based kernels: 0 default, 1 the alternative (N >= 4096)
#ifdef BCN_DEBUG
    bool debug = true;                 // device-side input checks before each call (bcn_ctx_set_debug)
#else
    bool debug = false;
#endif
    std::vector<uint64_t> primes;      // L data then K special
    // NTT twiddles per prime, [2N] interleaved (value, Shoup companion):
    // fwd[k] = psi^{brv(k)}, inv[k] = psi^{-brv(k)}; used by the host (client)
    // transforms and uploaded for the device ones
    std::vector<std::vector<uint32_t>> h_tw_fwd, h_tw_inv;
    // device tables
    bcn::PrimeConst *d_pc = nullptr;  // [P]
    uint2 *d_tw_fwd = nullptr;        // [P][N] (psi^{brv(k)}, shoup)
    uint2 *d_tw_inv = nullptr;        // [P][N] (psi^{-brv(k)}, shoup)
    uint32_t *d_ks = nullptr;         // KsTables blob
    uint32_t *d_status = nullptr;     // device status word (bounded waits that gave up)
    bcn::KsTables ks;
    std::vector<bcn::PrimeConst> h_pc;
};

// A linear layer as output groups: the outputs of a group read the same taps
// (one conv position with all its output channels; a whole dense layer).
struct bcn_layer_plan {
    int type, n_in, n_out, K, level, add, square;
    int in_ntt;                // the layer's inputs are in the NTT domain (a square layer came before)
    double s_w;
    int n_groups, n_go;        // groups, outputs per group
    int n_distinct_in;         // inputs the layer reads
    int32_t *d_gidx = nullptr; // [n_groups][K] input index per tap (-1: zero padding)
    int8_t *d_gw = nullptr;    // [n_groups][n_go][K]
    int32_t *d_gout = nullptr; // [n_groups][n_go] output index
    bcn::MacTcPlan tc;         // tensor-core MAC (tc.w16 == nullptr: not used)
};

namespace bcn {
// CUDA-event timing of the kernels an evaluation launches
struct Profiler {
    bool on = false;
    std::vector<cudaEvent_t> ev;
    size_t used = 0;
    struct Rec {
        int cls;
        size_t e0, e1;
        double bytes;
        int kernels;  // launches inside the timed scope
    };
    std::vector<Rec> recs;
    double ms[BCN_KERNEL_COUNT] = {};
    long long launches[BCN_KERNEL_COUNT] = {};
    double bytes[BCN_KERNEL_COUNT] = {};
};
}  // namespace bcn

struct bcn_model {
    bcn_ctx *ctx;
    std::vector<bcn_layer_plan> layers;
    mutable bcn::Profiler prof;
    int chunk;          // ciphertexts per key-switching chunk
    int chunk_request;  // 0: automatic
    int mac_impl = 0;   // 0: tensor cores where eligible, 1: CUDA cores only
    int overlap = 1;    // 1: a square layer's chunk halves and the feature transforms on extra streams
    int stack = 1;      // requests evaluated side by side (bcn_model_create_stacked)
    // copy streams of bcn_eval_host (created on first use) and, per workspace,
    // the event after the last evaluation that read its staged inputs; guarded
    // by copy_mu
    std::mutex copy_mu;
    std::vector<cudaStream_t> copy_streams;
    std::unordered_map<const void *, cudaEvent_t> staging_free;
    // second stream of bcn_eval's square layers (created on first use, guarded
    // by split_mu): a chunk's two halves run side by side
    std::mutex split_mu;
    cudaStream_t split_stream = nullptr;
    cudaStream_t aux_stream = nullptr;  // feature-plaintext transforms (also under split_mu)
    size_t ws_x_bytes;  // one ping-pong activation buffer
    size_t ws_y_bytes;  // MAC output of a square layer
    size_t ws_chunk_bytes;
    size_t ws_pt_bytes;  // NTT-domain copy of one layer's feature plaintexts
    int out_level;
};

namespace bcn {
// host <-> device glue implemented in the .cu files
bcn_status device_ctx_init(bcn_ctx *ctx);
void device_ctx_free(bcn_ctx *ctx);
void build_ks_tables(bcn_ctx *ctx);
}  // namespace bcn
