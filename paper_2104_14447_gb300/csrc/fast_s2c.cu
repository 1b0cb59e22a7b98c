// fast_s2c.cu -- instantiations of the warp-per-target stencil kernel: scalar 2D, degree 4.
// (Kernel in stencil_fast.cuh; split over several files so they compile in parallel.)
#include "stencil_fast.cuh"

namespace gmls {
extern const FastEntry kFastS2c[] = {GMLS_FAST(0, 2, 4, 2, 2, 32), GMLS_FAST(0, 2, 4, 2, 3, 32), GMLS_FAST(0, 2, 4, 3, 2, 32), GMLS_FAST(0, 2, 4, 3, 3, 32), GMLS_FAST(0, 2, 4, 3, 2, 16), GMLS_FAST(0, 2, 4, 3, 3, 16)};
extern const int kFastS2cCount = sizeof(kFastS2c) / sizeof(kFastS2c[0]);
}  // namespace gmls
