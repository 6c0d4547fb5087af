// NTT-based kernels for the small ring degrees N = 2^4 .. 2^11 (4 residues per thread).
#include "cores.cuh"

namespace bcn {
const CoreFns *core_fns_small(int logN) {
    switch (logN) {
    case 4: return CoreImpl<4, 4>::fns();
    case 5: return CoreImpl<5, 4>::fns();
    case 6: return CoreImpl<6, 4>::fns();
    case 7: return CoreImpl<7, 4>::fns();
    case 8: return CoreImpl<8, 4>::fns();
    case 9: return CoreImpl<9, 4>::fns();
    case 10: return CoreImpl<10, 4>::fns();
    case 11: return CoreImpl<11, 4>::fns();
    default: return nullptr;
    }
}
}  // namespace bcn
