// Square activation that allocates nothing.
//
// For callers that may not allocate device memory themselves: for example a
// serving process whose device memory is budgeted and handed out by an
// admission controller, or code running under a framework's caching allocator
// that forbids allocations behind its back (cudaMalloc and cudaFree also
// synchronise the device, which such callers must avoid mid-request).  The
// intermediates of the key switch live in one file-scope device array of
// kStaticScratchBytes; the caller passes only the inputs and outputs.
#include <mutex>

#include "device_api.h"

namespace bcn {
namespace {

constexpr size_t kStaticScratchBytes = 32ull << 20;  // 32 MiB, held by every GPU that loads the library
constexpr int kMaxDevices = 64;

static __device__ __align__(256) uint32_t g_scratch[kStaticScratchBytes / 4];

std::mutex g_mu;
uint32_t *g_scratch_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device, looked up once per
// device (the host-side name g_scratch is not a device address).
bcn_status scratch_address(int device, uint32_t **out) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (device < 0 || device >= kMaxDevices) return fail(BCN_E_INVAL, "device ordinal out of range");
    if (!g_scratch_addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || p == nullptr)
            return fail(BCN_E_CUDA, std::string("cudaGetSymbolAddress of the static scratch: ") +
                                        cudaGetErrorString(e));
        g_scratch_addr[device] = static_cast<uint32_t *>(p);
    }
    *out = g_scratch_addr[device];
    return BCN_OK;
}

}  // namespace
}  // namespace bcn

using namespace bcn;

extern "C" bcn_status bcn_op_square_relin_rescale_noalloc(const bcn_ctx *c, int level, const uint32_t *evk_eval,
                                                          const uint32_t *in, int n_ct, uint32_t *out,
                                                          void *stream) {
    if (!c) return fail(BCN_E_INVAL, "bcn_op_square_relin_rescale_noalloc: null ctx");
    if (c->device < 0) return fail(BCN_E_INVAL, "bcn_op_square_relin_rescale_noalloc: host-only ctx");
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess || cur != c->device)
        return fail(BCN_E_INVAL, "bcn_op_square_relin_rescale_noalloc: the ctx's device must be current");
    if (level < 2 || level > c->L) return fail(BCN_E_LEVEL, "bcn_op_square_relin_rescale_noalloc: level must be >= 2");
    if (!in || !out || !evk_eval || n_ct < 0 || ((uintptr_t)in & 15) || ((uintptr_t)out & 15) ||
        ((uintptr_t)evk_eval & 15))
        return fail(BCN_E_INVAL, "bcn_op_square_relin_rescale_noalloc: null, unaligned or negative argument");
    const size_t N = c->N, n = (size_t)level;
    const size_t d_words = 3 * n * N, acc_words = 2 * (n + c->K) * N;
    const size_t per_ct = (d_words + acc_words) * 4;
    const size_t chunk = kStaticScratchBytes / per_ct;
    if (chunk < 1)
        return fail(BCN_E_BUDGET, "bcn_op_square_relin_rescale_noalloc: one ciphertext at this level needs " +
                                      std::to_string(per_ct) + " bytes of scratch, the static scratch holds " +
                                      std::to_string(kStaticScratchBytes));
    uint32_t *scratch = nullptr;
    bcn_status s = scratch_address(c->device, &scratch);
    if (s != BCN_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    for (size_t o0 = 0; o0 < (size_t)n_ct; o0 += chunk) {
        const int C = (int)std::min(chunk, (size_t)n_ct - o0);
        uint32_t *d = scratch, *acc = scratch + (size_t)C * d_words;
        s = square_relin_rescale_chunk(c, level, evk_eval, in + o0 * 2 * n * N, d, acc, C,
                                       out + o0 * 2 * (n - 1) * N, st);
        if (s != BCN_OK) return s;
    }
    return BCN_OK;
}
