// NTT-based kernels for N = 2^12.
#include "cores.cuh"

#ifndef BCN_R12
#define BCN_R12 16  // residues per thread
#endif
#ifndef BCN_R12_KS
#define BCN_R12_KS BCN_R12  // key switch
#endif

namespace bcn {
const CoreFns *core_fns_12() { return CoreImpl<12, BCN_R12, BCN_R12_KS>::fns(); }
}  // namespace bcn
