// fast_d2.cu -- instantiations of the warp-per-target stencil kernel: divergence-free 2D, degrees 2-4 (vector Laplacian: 2 rows).
// (Kernel in stencil_fast.cuh; split over several files so they compile in parallel.)
#include "stencil_fast.cuh"

namespace gmls {
extern const FastEntry kFastD2[] = {GMLS_FAST(1, 2, 2, 2, 2, 32), GMLS_FAST(1, 2, 3, 3, 2, 32), GMLS_FAST(1, 2, 4, 3, 2, 32), GMLS_FAST(1, 2, 2, 3, 2, 16)};
extern const int kFastD2Count = sizeof(kFastD2) / sizeof(kFastD2[0]);
}  // namespace gmls
