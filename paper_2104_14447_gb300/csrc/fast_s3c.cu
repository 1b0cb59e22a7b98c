// fast_s3c.cu -- instantiations of the warp-per-target stencil kernel: scalar 3D, degree 4.
// (Kernel in stencil_fast.cuh; split over several files so they compile in parallel.)
#include "stencil_fast.cuh"

namespace gmls {
extern const FastEntry kFastS3c[] = {GMLS_FAST(0, 3, 4, 3, 4, 32), GMLS_FAST(0, 3, 4, 3, 3, 32)};
extern const int kFastS3cCount = sizeof(kFastS3c) / sizeof(kFastS3c[0]);
}  // namespace gmls
