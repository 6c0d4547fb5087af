// NTT-based kernels for N = 16384, the alternative block shape a context can
// select at run time (bcn_ctx_set_ntt_shape; the autotuner measures both):
// 16 residues per thread, 16 in the key switch.
#include "cores.cuh"

namespace bcn {
const CoreFns *core_fns_14_alt() { return CoreImpl<14, 16, 16>::fns(); }
}  // namespace bcn
