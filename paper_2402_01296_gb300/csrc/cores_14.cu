// NTT-based kernels for N = 2^14 (32 residues per thread).
#include "cores.cuh"

namespace bcn {
const CoreFns *core_fns_14() { return CoreImpl<14, 32>::fns(); }
}  // namespace bcn
