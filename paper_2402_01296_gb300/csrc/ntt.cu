// Batched negacyclic NTT / inverse NTT over RNS limbs (device).
//
// Forward: Cooley-Tukey with the 2N-th root psi merged into the twiddles
// (table psi^{brv(k)}), natural-order input, bit-reversed output; inverse:
// Gentleman-Sande with psi^{-brv(k)}, bit-reversed input, natural output,
// scaled by N^{-1}.  One thread block owns one limb; the limb sits in shared
// memory for all log N stages.  Twiddle products use Shoup multiplication.
#include <cuda_runtime.h>

#include "device_api.h"
#include "device_math.cuh"

namespace bcn {

__global__ void __launch_bounds__(512) k_ntt_fwd(uint32_t *__restrict__ data, int logN, PrimeMap pm,
                                                const PrimeConst *__restrict__ pc, const uint2 *__restrict__ tw) {
    extern __shared__ __align__(16) uint32_t s[];
    const int N = 1 << logN;
    const int limb = blockIdx.x;
    const int p = pm.pidx[limb % pm.period];
    const uint32_t q = pc[p].q;
    uint32_t *a = data + (size_t)limb * N;
    const uint2 *w = tw + (size_t)p * N;
    for (int i = threadIdx.x; i < N / 4; i += blockDim.x)
        reinterpret_cast<uint4 *>(s)[i] = reinterpret_cast<const uint4 *>(a)[i];
    __syncthreads();
    const int half = N >> 1;
    for (int m = 1, lt = logN - 1; m < N; m <<= 1, lt--) {
        const int t = 1 << lt;
        for (int b = threadIdx.x; b < half; b += blockDim.x) {
            const int i = b >> lt, j = b & (t - 1);
            const int x = (i << (lt + 1)) + j;
            const uint2 W = __ldg(&w[m + i]);
            const uint32_t U = s[x], V = shoup_mul(s[x + t], W.x, W.y, q);
            s[x] = add_mod(U, V, q);
            s[x + t] = sub_mod(U, V, q);
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < N / 4; i += blockDim.x)
        reinterpret_cast<uint4 *>(a)[i] = reinterpret_cast<const uint4 *>(s)[i];
}

__global__ void __launch_bounds__(512) k_ntt_inv(uint32_t *__restrict__ data, int logN, PrimeMap pm,
                                                const PrimeConst *__restrict__ pc, const uint2 *__restrict__ tw) {
    extern __shared__ __align__(16) uint32_t s[];
    const int N = 1 << logN;
    const int limb = blockIdx.x;
    const int p = pm.pidx[limb % pm.period];
    const uint32_t q = pc[p].q;
    uint32_t *a = data + (size_t)limb * N;
    const uint2 *w = tw + (size_t)p * N;
    for (int i = threadIdx.x; i < N / 4; i += blockDim.x)
        reinterpret_cast<uint4 *>(s)[i] = reinterpret_cast<const uint4 *>(a)[i];
    __syncthreads();
    const int half = N >> 1;
    for (int m = half, lt = 0; m >= 1; m >>= 1, lt++) {
        const int t = 1 << lt;
        for (int b = threadIdx.x; b < half; b += blockDim.x) {
            const int i = b >> lt, j = b & (t - 1);
            const int x = (i << (lt + 1)) + j;
            const uint2 W = __ldg(&w[m + i]);
            const uint32_t U = s[x], V = s[x + t];
            s[x] = add_mod(U, V, q);
            s[x + t] = shoup_mul(sub_mod(U, V, q), W.x, W.y, q);
        }
        __syncthreads();
    }
    const uint32_t ni = pc[p].ninv, nip = pc[p].ninv_shoup;
    for (int i = threadIdx.x; i < N / 4; i += blockDim.x) {
        uint4 v = reinterpret_cast<const uint4 *>(s)[i];
        v.x = shoup_mul(v.x, ni, nip, q);
        v.y = shoup_mul(v.y, ni, nip, q);
        v.z = shoup_mul(v.z, ni, nip, q);
        v.w = shoup_mul(v.w, ni, nip, q);
        reinterpret_cast<uint4 *>(a)[i] = v;
    }
}

bcn_status ntt_setup_kernels() {
    int smem = (1 << kMaxLogN) * 4;
    if (cudaFuncSetAttribute(k_ntt_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess ||
        cudaFuncSetAttribute(k_ntt_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return fail(BCN_E_CUDA, "cudaFuncSetAttribute failed for the NTT kernels");
    return BCN_OK;
}

bcn_status launch_ntt(const bcn_ctx *c, uint32_t *data, size_t n_limbs, const PrimeMap &pm, bool inverse,
                      cudaStream_t st) {
    if (n_limbs == 0) return BCN_OK;
    if (n_limbs > 0x7FFFFFFFull) return fail(BCN_E_INVAL, "too many limbs for one NTT launch");
    const int N = c->N;
    int threads = N / 2 < 512 ? N / 2 : 512;
    size_t smem = (size_t)N * 4;
    if (inverse)
        k_ntt_inv<<<(unsigned)n_limbs, threads, smem, st>>>(data, c->logN, pm, c->d_pc, c->d_tw_inv);
    else
        k_ntt_fwd<<<(unsigned)n_limbs, threads, smem, st>>>(data, c->logN, pm, c->d_pc, c->d_tw_fwd);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(BCN_E_CUDA, std::string("NTT launch: ") + cudaGetErrorString(e));
    return BCN_OK;
}

}  // namespace bcn
