// NTT-based kernels for N = 2^14.
#include "cores.cuh"

#ifndef BCN_R14
#define BCN_R14 16  // residues per thread
#endif

namespace bcn {
const CoreFns *core_fns_14() { return CoreImpl<14, BCN_R14>::fns(); }
}  // namespace bcn
