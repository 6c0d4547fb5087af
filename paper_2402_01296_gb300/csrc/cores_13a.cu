// NTT-based kernels for N = 8192, the alternative block shape a context can
// select at run time (bcn_ctx_set_ntt_shape; the autotuner measures both):
// 32 residues per thread, 32 in the key switch.
#include "cores.cuh"

namespace bcn {
const CoreFns *core_fns_13_alt() { return CoreImpl<13, 32, 32>::fns(); }
}  // namespace bcn
