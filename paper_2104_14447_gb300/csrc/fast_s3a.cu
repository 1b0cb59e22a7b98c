// fast_s3a.cu -- instantiations of the warp-per-target stencil kernel: scalar 3D, degree 2.
// (Kernel in stencil_fast.cuh; split over several files so they compile in parallel.)
#include "stencil_fast.cuh"

namespace gmls {
extern const FastEntry kFastS3a[] = {GMLS_FAST(0, 3, 2, 1, 3, 32), GMLS_FAST(0, 3, 2, 1, 4, 32), GMLS_FAST(0, 3, 2, 2, 3, 32), GMLS_FAST(0, 3, 2, 2, 4, 32), GMLS_FAST(0, 3, 2, 2, 3, 16), GMLS_FAST(0, 3, 2, 2, 4, 16)};
extern const int kFastS3aCount = sizeof(kFastS3a) / sizeof(kFastS3a[0]);
}  // namespace gmls
