// fast_s2b.cu -- instantiations of the warp-per-target stencil kernel: scalar 2D, degree 3.
// (Kernel in stencil_fast.cuh; split over several files so they compile in parallel.)
#include "stencil_fast.cuh"

namespace gmls {
extern const FastEntry kFastS2b[] = {GMLS_FAST(0, 2, 3, 1, 2, 32), GMLS_FAST(0, 2, 3, 1, 3, 32), GMLS_FAST(0, 2, 3, 2, 2, 32), GMLS_FAST(0, 2, 3, 2, 3, 32), GMLS_FAST(0, 2, 3, 2, 2, 16), GMLS_FAST(0, 2, 3, 2, 3, 16), GMLS_FAST(0, 2, 3, 3, 2, 16), GMLS_FAST(0, 2, 3, 3, 3, 16)};
extern const int kFastS2bCount = sizeof(kFastS2b) / sizeof(kFastS2b[0]);
}  // namespace gmls
