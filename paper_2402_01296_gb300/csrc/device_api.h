// Host-side launch helpers shared by the device translation units.
#pragma once

#include <cuda_runtime.h>

#include "bcn_internal.h"

namespace bcn {

bcn_status ntt_setup_kernels();
// In-place NTT of n_limbs consecutive limbs of N words; limb l uses prime
// pm.pidx[l % pm.period].
bcn_status launch_ntt(const bcn_ctx *c, uint32_t *data, size_t n_limbs, const PrimeMap &pm, bool inverse,
                      cudaStream_t st);

// prime map of a buffer whose limbs cycle through the data primes q_0..q_{level-1}
inline PrimeMap data_map(int level) {
    PrimeMap m{};
    m.period = level;
    for (int i = 0; i < level; i++) m.pidx[i] = (uint8_t)i;
    return m;
}
// prime map of the extended basis Q_level u P: q_0..q_{level-1}, p_0..p_{K-1}
inline PrimeMap ext_map(const bcn_ctx *c, int level) {
    PrimeMap m{};
    m.period = level + c->K;
    for (int i = 0; i < level; i++) m.pidx[i] = (uint8_t)i;
    for (int k = 0; k < c->K; k++) m.pidx[level + k] = (uint8_t)(c->L + k);
    return m;
}

inline bcn_status check_launch(const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(BCN_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    return BCN_OK;
}

}  // namespace bcn
