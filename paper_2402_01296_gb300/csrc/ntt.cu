// Dispatch of the NTT-based kernels by ring degree.
#include <algorithm>
#include <cuda_runtime.h>

#include "device_api.h"

namespace bcn {

const CoreFns *core_fns(int logN) {
    if (logN <= 11) return core_fns_small(logN);
    if (logN == 12) return core_fns_12();
    if (logN == 13) return core_fns_13();
    if (logN == 14) return core_fns_14();
    return nullptr;
}

bcn_status cores_setup_all() {
    for (int l = 4; l <= kMaxLogN; l++) {
        const CoreFns *f = core_fns(l);
        if (!f) return fail(BCN_E_INVAL, "unsupported ring degree");
        bcn_status s = f->setup();
        if (s != BCN_OK) return s;
    }
    return BCN_OK;
}

bcn_status launch_ntt_strided(const bcn_ctx *c, uint32_t *data, size_t n_limbs, size_t n_groups, size_t stride,
                              const PrimeMap &pm, bool inverse, cudaStream_t st) {
    const CoreFns *f = core_fns(c->logN);
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
