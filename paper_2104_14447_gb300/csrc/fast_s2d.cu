// fast_s2d.cu -- instantiations of the warp-per-target stencil kernel: scalar 2D, degree 4, 8-lane groups.
// (Kernel in stencil_fast.cuh; split over several files so they compile in parallel.)
#include "stencil_fast.cuh"

namespace gmls {
extern const FastEntry kFastS2d[] = {GMLS_FAST(0, 2, 4, 5, 2, 8), GMLS_FAST(0, 2, 4, 5, 3, 8)};
extern const int kFastS2dCount = sizeof(kFastS2d) / sizeof(kFastS2d[0]);
}  // namespace gmls
