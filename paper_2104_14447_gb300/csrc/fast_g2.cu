// fast_g2.cu -- instantiations of the warp-per-target stencil kernel: staggered 2D, degrees 2-4 (gradient and Laplacian: 3 rows).
// (Kernel in stencil_fast.cuh; split over several files so they compile in parallel.)
#include "stencil_fast.cuh"

namespace gmls {
extern const FastEntry kFastG2[] = {GMLS_FAST(2, 2, 2, 1, 3, 32), GMLS_FAST(2, 2, 2, 2, 3, 16),
                                    GMLS_FAST(2, 2, 3, 2, 3, 32), GMLS_FAST(2, 2, 3, 3, 3, 16),
                                    GMLS_FAST(2, 2, 4, 2, 3, 32), GMLS_FAST(2, 2, 4, 3, 3, 16)};
extern const int kFastG2Count = sizeof(kFastG2) / sizeof(kFastG2[0]);
}  // namespace gmls
