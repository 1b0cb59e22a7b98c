// fast_s3b.cu -- instantiations of the warp-per-target stencil kernel: scalar 3D, degree 3.
// (Kernel in stencil_fast.cuh; split over several files so they compile in parallel.)
#include "stencil_fast.cuh"

namespace gmls {
extern const FastEntry kFastS3b[] = {GMLS_FAST(0, 3, 3, 2, 3, 32), GMLS_FAST(0, 3, 3, 2, 4, 32), GMLS_FAST(0, 3, 3, 3, 3, 32), GMLS_FAST(0, 3, 3, 3, 4, 32), GMLS_FAST(0, 3, 3, 3, 3, 16), GMLS_FAST_T(0, 3, 3, 3, 4, 16, 384)};
extern const int kFastS3bCount = sizeof(kFastS3b) / sizeof(kFastS3b[0]);
}  // namespace gmls
