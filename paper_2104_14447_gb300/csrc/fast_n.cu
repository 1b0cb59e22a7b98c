// fast_n.cu -- Neumann instantiations of the warp-per-target stencil kernel:
// scalar basis with the constraint eliminated (boundary targets of the 3D
// degree-3 and 2D degree-4 operators: gradient and Laplacian rows).
// (Kernel in stencil_fast.cuh.)
#include "stencil_fast.cuh"

namespace gmls {
extern const FastEntry kFastN[] = {GMLS_FAST_NEU_T(3, 3, 3, 4, 16, 384), GMLS_FAST_NEU(3, 3, 2, 4, 32),
                                   GMLS_FAST_NEU(2, 4, 3, 3, 16), GMLS_FAST_NEU(2, 4, 2, 3, 32)};
extern const int kFastNCount = sizeof(kFastN) / sizeof(kFastN[0]);
}  // namespace gmls
