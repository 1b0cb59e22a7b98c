// fast_s2a.cu -- instantiations of the warp-per-target stencil kernel: scalar 2D, degree 2.
// (Kernel in stencil_fast.cuh; split over several files so they compile in parallel.)
#include "stencil_fast.cuh"

namespace gmls {
extern const FastEntry kFastS2a[] = {GMLS_FAST(0, 2, 2, 1, 2, 32), GMLS_FAST(0, 2, 2, 1, 3, 32), GMLS_FAST(0, 2, 2, 2, 2, 32), GMLS_FAST(0, 2, 2, 2, 3, 32), GMLS_FAST(0, 2, 2, 1, 2, 16), GMLS_FAST(0, 2, 2, 1, 3, 16), GMLS_FAST(0, 2, 2, 2, 2, 16), GMLS_FAST(0, 2, 2, 2, 3, 16)};
extern const int kFastS2aCount = sizeof(kFastS2a) / sizeof(kFastS2a[0]);
}  // namespace gmls
