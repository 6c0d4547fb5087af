// NTT-based kernels for N = 2^12 (16 residues per thread).
#include "cores.cuh"

namespace bcn {
const CoreFns *core_fns_12() { return CoreImpl<12, 16>::fns(); }
}  // namespace bcn
