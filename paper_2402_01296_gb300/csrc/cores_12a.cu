// NTT-based kernels for N = 4096, the alternative block shape a context can
// select at run time (bcn_ctx_set_ntt_shape; the autotuner measures both):
// 8 residues per thread, 8 in the key switch.
#include "cores.cuh"

namespace bcn {
const CoreFns *core_fns_12_alt() { return CoreImpl<12, 8, 8>::fns(); }
}  // namespace bcn
