// NTT-based kernels for N = 2^13.
#include "cores.cuh"

#ifndef BCN_R13
#define BCN_R13 16  // residues per thread
#endif
#ifndef BCN_R13_KS
#define BCN_R13_KS BCN_R13  // key switch
#endif

namespace bcn {
const CoreFns *core_fns_13() { return CoreImpl<13, BCN_R13, BCN_R13_KS>::fns(); }
}  // namespace bcn
