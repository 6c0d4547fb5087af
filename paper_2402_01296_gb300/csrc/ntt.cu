// Dispatch of the NTT-based kernels by ring degree.
#include <algorithm>
#include <cuda_runtime.h>

#include "device_api.h"

namespace bcn {

// alt: the alternative block shape of N = 4096, 8192, 16384 (cores_1Xa.cu);
// smaller rings have one shape
const CoreFns *core_fns(int logN, int alt) {
    if (logN <= 11) return core_fns_small(logN);
    if (logN == 12) return alt ? core_fns_12_alt() : core_fns_12();
    if (logN == 13) return alt ? core_fns_13_alt() : core_fns_13();
    if (logN == 14) return alt ? core_fns_14_alt() : core_fns_14();
    return nullptr;
}

const CoreFns *core_fns(const bcn_ctx *c) { return core_fns(c->logN, c->ntt_alt); }

bcn_status cores_setup_all() {
    for (int l = 4; l <= kMaxLogN; l++)
        for (int alt = 0; alt < (l >= 12 ? 2 : 1); alt++) {
            const CoreFns *f = core_fns(l, alt);
            if (!f) return fail(BCN_E_INVAL, "unsupported ring degree");
            bcn_status s = f->setup();
            if (s != BCN_OK) return s;
        }
    return BCN_OK;
}

bcn_status launch_ntt_strided(const bcn_ctx *c, uint32_t *data, size_t n_limbs, size_t n_groups, size_t stride,
                              const PrimeMap &pm, bool inverse, cudaStream_t st) {
    const CoreFns *f = core_fns(c);
    if (!f) return fail(BCN_E_INVAL, "unsupported ring degree");
    for (size_t g0 = 0; g0 < n_groups; g0 += 65535) {  // grid.y limit
        const size_t G = std::min<size_t>(65535, n_groups - g0);
        bcn_status s = f->ntt(c, data + g0 * stride, n_limbs, G, stride, pm, inverse, st);
        if (s != BCN_OK) return s;
    }
    return BCN_OK;
}

bcn_status launch_ntt(const bcn_ctx *c, uint32_t *data, size_t n_limbs, const PrimeMap &pm, bool inverse,
                      cudaStream_t st) {
    if (n_limbs == 0) return BCN_OK;
    if (n_limbs > 0x7FFFFFFFull) return fail(BCN_E_INVAL, "too many limbs for one NTT launch");
    return launch_ntt_strided(c, data, n_limbs, 1, 0, pm, inverse, st);
}

}  // namespace bcn

using namespace bcn;

// residues per thread of the NTT and square kernels of a shape (the key switch
// of the alternative shapes uses the same)
static int shape_r(int logN, int alt) {
    if (logN <= 11) return -1;
    static const int def[3] = {16, 16, 32}, other[3] = {8, 32, 16};
    return alt ? other[logN - 12] : def[logN - 12];
}

extern "C" bcn_status bcn_ctx_set_ntt_shape(bcn_ctx *c, int alt) {
    if (!c || (alt != 0 && alt != 1)) return fail(BCN_E_INVAL, "bcn_ctx_set_ntt_shape: shape 0 or 1");
    if (alt && c->logN < 12) return fail(BCN_E_INVAL, "bcn_ctx_set_ntt_shape: one shape below N = 4096");
    c->ntt_alt = alt;
    return BCN_OK;
}

extern "C" bcn_status bcn_ctx_get_ntt_shape(const bcn_ctx *c, int *alt, int *residues_per_thread) {
    if (!c || !alt) return fail(BCN_E_INVAL, "bcn_ctx_get_ntt_shape: null argument");
    *alt = c->ntt_alt;
    if (residues_per_thread) *residues_per_thread = shape_r(c->logN, c->ntt_alt);
    return BCN_OK;
}
