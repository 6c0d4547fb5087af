// NTT-based kernels for N = 2^13 (16 residues per thread).
#include "cores.cuh"

namespace bcn {
const CoreFns *core_fns_13() { return CoreImpl<13, 16>::fns(); }
}  // namespace bcn
