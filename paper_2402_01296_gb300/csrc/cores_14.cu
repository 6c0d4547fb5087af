// NTT-based kernels for N = 2^14.
#include "cores.cuh"

#ifndef BCN_R14
#define BCN_R14 32  // residues per thread: NTT and square kernels (512 threads; the square kernel on
                    // coefficient input at 128 registers: 12.0 against 15.7 ms per CIFAR-shaped
                    // evaluation with 16 residues and 1024 threads)
#endif
#ifndef BCN_R14_KS
#define BCN_R14_KS 32  // key switch: two groups of 16 per pass (512 threads, 128 registers)
#endif

namespace bcn {
const CoreFns *core_fns_14() { return CoreImpl<14, BCN_R14, BCN_R14_KS>::fns(); }
}  // namespace bcn
