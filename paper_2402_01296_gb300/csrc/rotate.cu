// Slot rotation (App. A: D(Rot(c, k)) is D(c) rotated by k slots; App. D
// builds packed convolutions and dense layers from rotations).
//
// With slot k at the root zeta^{5^k}, the rotation by r slots is the
// automorphism sigma_g: a(X) -> a(X^g), g = 5^r mod 2N, followed by key
// switching from sigma_g(s) back to s with the Galois key of g:
//     Rot(c0, c1) = (sigma_g(c0) + k0, k1),  (k0, k1) = KeySwitch_gk(sigma_g(c1)).
// Per chunk of ciphertexts: sigma_g(c1) into the key-switching input, the fused
// key-switching core (ModUp, NTT, key product, iNTT -- the same kernel as the
// relinearisation), then ModDown with sigma_g(c0) added (no rescale).
#include <algorithm>
#include <string>
#include <cuda_runtime.h>

#include "device_api.h"
#include "device_math.cuh"

namespace bcn {
namespace {

// coefficient j of a(X^g): a_i with i = j g^{-1} mod 2N when i < N, else
// -a_{i-N} (X^N = -1); ginv = g^{-1} mod 2N, N a power of two
__device__ __forceinline__ uint32_t auto_coeff(const uint32_t *__restrict__ a, int j, uint32_t ginv, int N,
                                               uint32_t q) {
    const uint32_t i = (uint32_t)(((uint64_t)j * ginv) & (uint64_t)(2 * N - 1));
    if (i < (uint32_t)N) return __ldg(a + i);
    const uint32_t v = __ldg(a + (i - N));
    return v ? q - v : 0u;
}

// D [C][3][n][N] slot 2 <- sigma_g(c1) of in [C][2][n][N].  grid (N/256, n, C)
__global__ void __launch_bounds__(256) k_automorph_c1(const uint32_t *__restrict__ in, uint32_t *__restrict__ D,
                                                      int n, int N, uint32_t ginv,
                                                      const PrimeConst *__restrict__ pc) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    const int i = blockIdx.y, ct = blockIdx.z;
    const uint32_t *a = in + (((size_t)ct * 2 + 1) * n + i) * N;
    D[(((size_t)ct * 3 + 2) * n + i) * N + j] = auto_coeff(a, j, ginv, N, pc[i].q);
}

// ModDown by P of the key-switching sums of one poly b (acc [n+K][N], centred
// fast basis conversion of the P part), plus sigma_g(c0) (c0 [n][N], the
// rotated ciphertext's first poly) when b == 0: out [n][N].  Coefficients
// 4 k4 .. 4 k4 + 3.
__device__ __forceinline__ void moddown_rotate_body(const uint32_t *__restrict__ c0_base,
                                                    const uint32_t *__restrict__ acc_b, uint32_t *__restrict__ out_b,
                                                    int b, int n, int N, uint32_t ginv, const KsDev &ks,
                                                    const PrimeConst *__restrict__ pc, int k4) {
    const int L = ks.L;
    const uint4 *ab = reinterpret_cast<const uint4 *>(acc_b) + k4;
    uint4 *ob = reinterpret_cast<uint4 *>(out_b) + k4;
    const size_t stride = (size_t)N / 4;
    uint32_t r[4][4];  // [special prime][coefficient]
    int cnt[4] = {0, 0, 0, 0};
#pragma unroll
    for (int m = 0; m < 4; m++) {  // K <= 4
        if (m >= ks.K) break;
        const PrimeConst &pm = pc[L + m];
        // a_m Phat_m^{-1}: the prepared key's special-prime limbs carry Phat_m^{-1}
        const uint4 v = __ldg(ab + (size_t)(n + m) * stride);
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int z = 0; z < 4; z++) {
            r[m][z] = w[z];
            cnt[z] += r[m][z] > pm.half;
        }
    }
    for (int i = 0; i < n; i++) {
        const uint32_t q = pc[i].q;
        uint32_t conv[4] = {0, 0, 0, 0};
#pragma unroll
        for (int m = 0; m < 4; m++) {
            if (m >= ks.K) break;
            const uint2 ph = ks.phat[(size_t)m * L + i];
#pragma unroll
            for (int z = 0; z < 4; z++) conv[z] = add_mod(conv[z], shoup_mul(r[m][z], ph.x, ph.y, q), q);
        }
        const uint32_t pmod = ks.pmod[i];
        const uint2 pi = ks.pinv[i];
        const uint4 av = __ldg(ab + (size_t)i * stride);
        const uint32_t a[4] = {av.x, av.y, av.z, av.w};
        const uint32_t *c0 = c0_base + (size_t)i * N;
        uint32_t o[4];
#pragma unroll
        for (int z = 0; z < 4; z++) {
            for (int c = 0; c < cnt[z]; c++) conv[z] = sub_mod(conv[z], pmod, q);
            const uint32_t kv = shoup_mul(sub_mod(a[z], conv[z], q), pi.x, pi.y, q);
            o[z] = b == 0 ? add_mod(kv, auto_coeff(c0, 4 * k4 + z, ginv, N, q), q) : kv;
        }
        ob[(size_t)i * stride] = make_uint4(o[0], o[1], o[2], o[3]);
    }
}

// ModDown + sigma_g(c0) of one rotation of C ciphertexts: ACC [C][2][n+K][N]
// -> out [C][2][n][N].  grid (N/4/256, 2, C)
__global__ void __launch_bounds__(256) k_moddown_rotate(const uint32_t *__restrict__ in,
                                                        const uint32_t *__restrict__ acc,
                                                        uint32_t *__restrict__ out, int n, int N, uint32_t ginv,
                                                        KsDev ks, const PrimeConst *__restrict__ pc) {
    const int k4 = blockIdx.x * blockDim.x + threadIdx.x;
    if (k4 * 4 >= N) return;
    const int b = blockIdx.y, ct = blockIdx.z, nb = n + ks.K;
    moddown_rotate_body(in + (size_t)ct * 2 * n * N, acc + ((size_t)ct * 2 + b) * nb * N,
                        out + ((size_t)ct * 2 + b) * n * N, b, n, N, ginv, ks, pc, k4);
}

// The same for a batch of rotations of C ciphertexts: ACC [C][count][2][n+K][N]
// (k_ks_rot) -> out [n_ct_total][n_rot_total][2][n][N] at ciphertext ct0 + ct,
// rotation r0 + r.  grid (N/4/256, 2 * count, C)
__global__ void __launch_bounds__(256) k_moddown_rot_many(const uint32_t *__restrict__ in,
                                                          const uint32_t *__restrict__ acc,
                                                          uint32_t *__restrict__ out, int n, int N, RotBatch rb,
                                                          int n_rot_total, int r0, KsDev ks,
                                                          const PrimeConst *__restrict__ pc) {
    const int k4 = blockIdx.x * blockDim.x + threadIdx.x;
    if (k4 * 4 >= N) return;
    const int b = blockIdx.y & 1, r = blockIdx.y >> 1, ct = blockIdx.z, nb = n + ks.K;
    const size_t ct_words = (size_t)2 * n * N;
    moddown_rotate_body(in + (size_t)ct * ct_words, acc + (((size_t)ct * rb.count + r) * 2 + b) * nb * N,
                        out + ((size_t)ct * n_rot_total + r0 + r) * ct_words + (size_t)b * n * N, b, n, N,
                        rb.ginv[r], ks, pc, k4);
}

// Sum of products in the NTT domain: out[b][i][k] = sum_r R[r][b][i][k] U[r][i][k]
// mod q_i (R [n_terms][2][n][N] the rotated ciphertexts, U [n_terms][n][N] the
// diagonal plaintexts, both canonical), added to out's own values when
// `accumulate` is set.  Products below 2^60 summed in 64 bits, reduced every 15
// terms (the first group of 15 also holds out's value, below 2^32).  Four coefficients a thread.  grid (N/4/256, n, 2)
__global__ void __launch_bounds__(256) k_mul_acc(const uint32_t *__restrict__ R, const uint32_t *__restrict__ U,
                                                 uint32_t *__restrict__ out, int n_terms, int n, int N,
                                                 int accumulate, const PrimeConst *__restrict__ pc) {
    const int k4 = blockIdx.x * blockDim.x + threadIdx.x;
    if (k4 * 4 >= N) return;
    const int i = blockIdx.y, b = blockIdx.z;
    const uint32_t q = pc[i].q;
    const uint64_t mu = pc[i].barrett;
    const size_t ct_words = (size_t)2 * n * N;
    uint64_t acc[4] = {0, 0, 0, 0};
    if (accumulate) {  // add to the running sum of earlier inputs (canonical, < 2^32)
        const uint4 o = reinterpret_cast<const uint4 *>(out + ((size_t)b * n + i) * N)[k4];
        acc[0] = o.x, acc[1] = o.y, acc[2] = o.z, acc[3] = o.w;
    }
    int cnt = 0;
    for (int r = 0; r < n_terms; r++) {
        const uint4 x = __ldg(reinterpret_cast<const uint4 *>(R + r * ct_words + ((size_t)b * n + i) * N) + k4);
        const uint4 u = __ldg(reinterpret_cast<const uint4 *>(U + ((size_t)r * n + i) * N) + k4);
        acc[0] += (uint64_t)x.x * u.x;
        acc[1] += (uint64_t)x.y * u.y;
        acc[2] += (uint64_t)x.z * u.z;
        acc[3] += (uint64_t)x.w * u.w;
        if (++cnt == 15) {
#pragma unroll
            for (int z = 0; z < 4; z++) acc[z] = barrett_reduce64(acc[z], q, mu);
            cnt = 0;
        }
    }
    uint4 o;
    o.x = barrett_reduce64(acc[0], q, mu);
    o.y = barrett_reduce64(acc[1], q, mu);
    o.z = barrett_reduce64(acc[2], q, mu);
    o.w = barrett_reduce64(acc[3], q, mu);
    reinterpret_cast<uint4 *>(out + ((size_t)b * n + i) * N)[k4] = o;
}

// Add(c, u) of App. A for a plaintext per ciphertext: c0 += u mod q_i, in place
// (ct [C][2][n][N], pt [C][n][N], coefficient form, canonical).  Four
// coefficients a thread.  grid (N/4/256, n, C)
__global__ void __launch_bounds__(256) k_add_plain(uint32_t *__restrict__ ct, const uint32_t *__restrict__ pt, int n,
                                                   int N, const PrimeConst *__restrict__ pc) {
    const int k4 = blockIdx.x * blockDim.x + threadIdx.x;
    if (k4 * 4 >= N) return;
    const int i = blockIdx.y, g = blockIdx.z;
    const uint32_t q = pc[i].q;
    uint4 *c = reinterpret_cast<uint4 *>(ct + ((size_t)g * 2 * n + i) * N) + k4;
    const uint4 u = __ldg(reinterpret_cast<const uint4 *>(pt + ((size_t)g * n + i) * N) + k4);
    uint4 v = *c;
    v.x = add_mod(v.x, u.x, q);
    v.y = add_mod(v.y, u.y, q);
    v.z = add_mod(v.z, u.z, q);
    v.w = add_mod(v.w, u.w, q);
    *c = v;
}

// g^{-1} mod 2N: the odd residues mod 2N form a group of order N, so g^{N-1}
static uint64_t galois_inverse(uint64_t g, uint64_t N) {
    const uint64_t two_n = 2 * N;
    uint64_t ginv = 1, base = g % two_n;
    for (uint64_t e = N - 1; e; e >>= 1) {
        if (e & 1) ginv = ginv * base % two_n;
        base = base * base % two_n;
    }
    return ginv;
}

// ciphertexts per hoisted-rotation chunk: U and one rotation batch's sums per
// ciphertext (words)
static size_t hoist_words_per_ct(const bcn_ctx *c, int n) {
    const size_t nb = (size_t)n + c->K, dnum = ((size_t)n + c->alpha - 1) / c->alpha;
    return (dnum * nb + (size_t)kRotBatch * 2 * nb) * c->N;
}
constexpr int kHoistChunk = 8;

}  // namespace
}  // namespace bcn

using namespace bcn;

extern "C" bcn_status bcn_op_rotate_many_workspace_bytes(const bcn_ctx *c, int level, int n_ct, size_t *bytes) {
    if (!c || !bytes || level < 1 || level > c->L || n_ct < 0) return fail(BCN_E_INVAL, "bad argument");
    const size_t chunk = (size_t)std::min(std::max(n_ct, 1), kHoistChunk);
    *bytes = chunk * hoist_words_per_ct(c, level) * 4;
    return BCN_OK;
}

extern "C" bcn_status bcn_op_rotate_many(const bcn_ctx *c, int level, const uint32_t *const *gk_evals,
                                         const int *steps, int n_rot, const uint32_t *in, int n_ct, uint32_t *out,
                                         void *ws, size_t ws_bytes, void *stream) {
    if (!c) return fail(BCN_E_INVAL, "bcn_op_rotate_many: null context");
    if (c->device < 0) return fail(BCN_E_INVAL, "bcn_op_rotate_many: host-only ctx");
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess || cur != c->device)
        return fail(BCN_E_INVAL, "bcn_op_rotate_many: the ctx's device must be current");
    if (level < 1 || level > c->L || n_ct < 0 || n_rot < 0 || c->K < 1)
        return fail(BCN_E_INVAL, "bcn_op_rotate_many: bad level or count");
    if (n_ct == 0 || n_rot == 0) return BCN_OK;
    if (!gk_evals || !steps) return fail(BCN_E_INVAL, "bcn_op_rotate_many: null key or step array");
    size_t need = 0;
    BCN_TRY(bcn_op_rotate_many_workspace_bytes(c, level, n_ct, &need));
    if (!ws || ws_bytes < need) return fail(BCN_E_BUDGET, "bcn_op_rotate_many: workspace too small");
    auto a16 = [](const void *p) { return ((uintptr_t)p & 15) == 0; };
    if (!in || !out || !a16(in) || !a16(out) || !a16(ws))
        return fail(BCN_E_INVAL, "bcn_op_rotate_many: null or unaligned buffer");
    const size_t N = c->N, n = (size_t)level, ct_words = 2 * n * N;
    const uint32_t *in_end = in + (size_t)n_ct * ct_words, *out_end = out + (size_t)n_ct * n_rot * ct_words;
    if (in < out_end && out < in_end) return fail(BCN_E_INVAL, "bcn_op_rotate_many: in and out overlap");
    const uint32_t half = (uint32_t)(N / 2);
    for (int r = 0; r < n_rot; r++) {
        const uint32_t s = (uint32_t)(((long long)steps[r] % (long long)half + half) % half);
        if (s != 0 && (!gk_evals[r] || !a16(gk_evals[r])))
            return fail(BCN_E_INVAL, "bcn_op_rotate_many: missing or unaligned Galois key");
    }
    const CoreFns *f = core_fns(c);
    if (!f) return fail(BCN_E_INVAL, "unsupported ring degree");
    cudaStream_t st = (cudaStream_t)stream;
    BCN_TRY(debug_check_input(c, in, 2 * (size_t)n_ct, level, st, "bcn_op_rotate_many"));
    const size_t nb = n + c->K, dnum = (n + c->alpha - 1) / c->alpha;
    const int chunk = std::min(n_ct, kHoistChunk);
    uint32_t *U = reinterpret_cast<uint32_t *>(ws);
    uint32_t *acc = U + (size_t)chunk * dnum * nb * N;
    for (int o0 = 0; o0 < n_ct; o0 += chunk) {
        const int C = std::min(chunk, n_ct - o0);
        const uint32_t *x = in + (size_t)o0 * ct_words;
        bool any = false;
        for (int r = 0; r < n_rot; r++) {  // identity rotations are copies
            const uint32_t s = (uint32_t)(((long long)steps[r] % (long long)half + half) % half);
            if (s != 0) {
                any = true;
                continue;
            }
            for (int k = 0; k < C; k++)
                if (cudaMemcpyAsync(out + ((size_t)(o0 + k) * n_rot + r) * ct_words, x + (size_t)k * ct_words,
                                    ct_words * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
                    return fail(BCN_E_CUDA, "bcn_op_rotate_many: copy failed");
        }
        if (!any) continue;
        BCN_TRY(f->modup_hoist(c, level, x, U, C, st));
        RotBatch rb;
        rb.count = 0;
        int r0 = -1;
        // gather the non-identity rotations into batches of consecutive indices
        auto flush = [&]() -> bcn_status {
            if (rb.count == 0) return BCN_OK;
            BCN_TRY(f->ks_rot(c, level, U, rb, acc, C, st));
            k_moddown_rot_many<<<dim3((unsigned)((N / 4 + 255) / 256), 2 * rb.count, C), 256, 0, st>>>(
                x, acc, out + (size_t)o0 * n_rot * ct_words, level, (int)N, rb, n_rot, r0, ks_dev(c), c->d_pc);
            BCN_TRY(check_launch("k_moddown_rot_many"));
            rb.count = 0;
            r0 = -1;
            return BCN_OK;
        };
        for (int r = 0; r < n_rot; r++) {
            const uint32_t s = (uint32_t)(((long long)steps[r] % (long long)half + half) % half);
            if (s == 0 || (r0 >= 0 && r != r0 + rb.count) || rb.count == kRotBatch) BCN_TRY(flush());
            if (s == 0) continue;
            if (r0 < 0) r0 = r;
            const uint64_t g = bcn_galois_elt(c, (int)s);
            rb.gk[rb.count] = gk_evals[r];
            rb.g[rb.count] = (uint32_t)g;
            rb.ginv[rb.count] = (uint32_t)galois_inverse(g, N);
            rb.count++;
        }
        BCN_TRY(flush());
    }
    return BCN_OK;
}

extern "C" bcn_status bcn_op_fc_diag_workspace_bytes(const bcn_ctx *c, int level, int n_rot, size_t *bytes) {
    if (!c || !bytes || level < 2 || level > c->L || n_rot < 1) return fail(BCN_E_INVAL, "bad argument");
    size_t rot = 0;
    BCN_TRY(bcn_op_rotate_many_workspace_bytes(c, level, 1, &rot));
    const size_t ct_bytes = (size_t)2 * level * c->N * 4;
    *bytes = rot + (size_t)n_rot * ct_bytes + ct_bytes;
    return BCN_OK;
}

// Diagonal-method dense layer over n_in input ciphertexts per group, summed
// before the one inverse transform and rescale, then the optional plaintext
// added (bcn_op_fc_diag is n_in = 1, no plaintext).
static bcn_status fc_diag_impl(const bcn_ctx *c, const char *who, int level, const uint32_t *const *gk_evals,
                               const int *steps, int n_rot, const uint32_t *diag_ntt, const uint32_t *in, int n_in,
                               int n_groups, const uint32_t *pt, uint32_t *out, void *ws, size_t ws_bytes,
                               void *stream) {
    if (!c) return fail(BCN_E_INVAL, std::string(who) + ": null context");
    if (level < 2 || level > c->L || n_groups < 0 || n_rot < 1 || n_in < 1)
        return fail(BCN_E_INVAL, std::string(who) + ": bad level or count");
    if (n_groups == 0) return BCN_OK;
    size_t need = 0;
    BCN_TRY(bcn_op_fc_diag_workspace_bytes(c, level, n_rot, &need));
    if (!ws || ws_bytes < need) return fail(BCN_E_BUDGET, std::string(who) + ": workspace too small");
    auto a16 = [](const void *p) { return ((uintptr_t)p & 15) == 0; };
    if (!diag_ntt || !in || !out || !a16(diag_ntt) || !a16(in) || !a16(out) || !a16(ws) || (pt && !a16(pt)))
        return fail(BCN_E_INVAL, std::string(who) + ": null or unaligned buffer");
    const size_t N = c->N, n = (size_t)level, ct_words = 2 * n * N, out_words = 2 * (n - 1) * N;
    const uint32_t *in_end = in + (size_t)n_groups * n_in * ct_words, *out_end = out + (size_t)n_groups * out_words;
    if (in < out_end && out < in_end) return fail(BCN_E_INVAL, std::string(who) + ": in and out overlap");
    size_t rot_bytes = 0;
    BCN_TRY(bcn_op_rotate_many_workspace_bytes(c, level, 1, &rot_bytes));
    char *w = reinterpret_cast<char *>(ws);
    uint32_t *R = reinterpret_cast<uint32_t *>(w + rot_bytes);
    uint32_t *acc = R + (size_t)n_rot * ct_words;
    cudaStream_t st = (cudaStream_t)stream;
    BCN_TRY(debug_check_input(c, in, 2 * (size_t)n_groups * n_in, level, st, who));
    if (pt) BCN_TRY(debug_check_input(c, pt, (size_t)n_groups, level - 1, st, who));
    const dim3 grid((unsigned)((N / 4 + 255) / 256), (unsigned)n, 2);
    for (int g = 0; g < n_groups; g++) {
        for (int k = 0; k < n_in; k++) {
            const uint32_t *x = in + ((size_t)g * n_in + k) * ct_words;
            BCN_TRY(bcn_op_rotate_many(c, level, gk_evals, steps, n_rot, x, 1, R, ws, rot_bytes, stream));
            BCN_TRY(launch_ntt(c, R, (size_t)n_rot * 2 * n, data_map(level), false, st));
            k_mul_acc<<<grid, 256, 0, st>>>(R, diag_ntt + (size_t)k * n_rot * n * N, acc, n_rot, level, (int)N,
                                            k > 0, c->d_pc);
            BCN_TRY(check_launch("k_mul_acc"));
        }
        uint32_t *o = out + (size_t)g * out_words;
        BCN_TRY(launch_ntt(c, acc, 2 * n, data_map(level), true, st));
        BCN_TRY(launch_rescale(c, level, acc, o, 1, st));
        if (pt) {
            k_add_plain<<<dim3((unsigned)((N / 4 + 255) / 256), (unsigned)(n - 1), 1), 256, 0, st>>>(
                o, pt + (size_t)g * (n - 1) * N, (int)(n - 1), (int)N, c->d_pc);
            BCN_TRY(check_launch("k_add_plain"));
        }
    }
    return BCN_OK;
}

extern "C" bcn_status bcn_op_fc_diag(const bcn_ctx *c, int level, const uint32_t *const *gk_evals, const int *steps,
                                     int n_rot, const uint32_t *diag_ntt, const uint32_t *in, int n_ct,
                                     uint32_t *out, void *ws, size_t ws_bytes, void *stream) {
    return fc_diag_impl(c, "bcn_op_fc_diag", level, gk_evals, steps, n_rot, diag_ntt, in, 1, n_ct, nullptr, out, ws,
                        ws_bytes, stream);
}

extern "C" bcn_status bcn_op_fc_diag_sum(const bcn_ctx *c, int level, const uint32_t *const *gk_evals,
                                         const int *steps, int n_rot, const uint32_t *diag_ntt, const uint32_t *in,
                                         int n_in, int n_groups, const uint32_t *pt, uint32_t *out, void *ws,
                                         size_t ws_bytes, void *stream) {
    return fc_diag_impl(c, "bcn_op_fc_diag_sum", level, gk_evals, steps, n_rot, diag_ntt, in, n_in, n_groups, pt, out,
                        ws, ws_bytes, stream);
}

extern "C" bcn_status bcn_op_rotate(const bcn_ctx *c, int level, const uint32_t *gk, int steps, const uint32_t *in,
                                    int n_ct, uint32_t *out, void *ws, size_t ws_bytes, void *stream) {
    if (!c) return fail(BCN_E_INVAL, "bcn_op_rotate: null context");
    if (c->device < 0) return fail(BCN_E_INVAL, "bcn_op_rotate: host-only ctx");
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess || cur != c->device)
        return fail(BCN_E_INVAL, "bcn_op_rotate: the ctx's device must be current");
    if (level < 1 || level > c->L || n_ct < 0 || c->K < 1) return fail(BCN_E_INVAL, "bcn_op_rotate: bad level");
    if (n_ct == 0) return BCN_OK;
    size_t need = 0;
    BCN_TRY(bcn_op_workspace_bytes(c, level, n_ct, &need));
    if (!ws || ws_bytes < need) return fail(BCN_E_BUDGET, "bcn_op_rotate: workspace too small");
    auto a16 = [](const void *p) { return ((uintptr_t)p & 15) == 0; };
    if (!gk || !in || !out || !a16(gk) || !a16(in) || !a16(out) || !a16(ws))
        return fail(BCN_E_INVAL, "bcn_op_rotate: null or unaligned buffer");
    const size_t N = c->N, ct_words = 2 * (size_t)level * N;
    const uint32_t *in_end = in + (size_t)n_ct * ct_words, *out_end = out + (size_t)n_ct * ct_words;
    if (in < out_end && out < in_end) return fail(BCN_E_INVAL, "bcn_op_rotate: in and out overlap");
    const CoreFns *f = core_fns(c);
    if (!f) return fail(BCN_E_INVAL, "unsupported ring degree");
    const uint64_t g = bcn_galois_elt(c, steps), ginv = galois_inverse(g, N);
    cudaStream_t st = (cudaStream_t)stream;
    BCN_TRY(debug_check_input(c, in, 2 * (size_t)n_ct, level, st, "bcn_op_rotate"));
    const int n = level, chunk = ks_default_chunk(c, level, n_ct);
    uint32_t *d, *d2n, *acc;
    ks_carve(c, n, chunk, reinterpret_cast<char *>(ws), &d, &d2n, &acc);
    for (int o0 = 0; o0 < n_ct; o0 += chunk) {
        const int C = std::min(chunk, n_ct - o0);
        const uint32_t *x = in + (size_t)o0 * ct_words;
        k_automorph_c1<<<dim3((unsigned)((N + 255) / 256), n, C), 256, 0, st>>>(x, d, n, (int)N, (uint32_t)ginv,
                                                                             c->d_pc);
        BCN_TRY(check_launch("k_automorph_c1"));
        BCN_TRY(f->keyswitch(c, n, d, nullptr, gk, acc, C, false, st));
        k_moddown_rotate<<<dim3((unsigned)((N / 4 + 255) / 256), 2, C), 256, 0, st>>>(
            x, acc, out + (size_t)o0 * ct_words, n, (int)N, (uint32_t)ginv, ks_dev(c), c->d_pc);
        BCN_TRY(check_launch("k_moddown_rotate"));
    }
    return BCN_OK;
}
