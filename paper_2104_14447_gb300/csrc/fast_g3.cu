// fast_g3.cu -- instantiations of the warp-per-target stencil kernel: staggered 3D, degree 2 (gradient and Laplacian: 4 rows).
// (Kernel in stencil_fast.cuh; split over several files so they compile in parallel.)
#include "stencil_fast.cuh"

namespace gmls {
extern const FastEntry kFastG3[] = {GMLS_FAST(2, 3, 2, 2, 4, 32), GMLS_FAST(2, 3, 2, 3, 4, 16)};
extern const int kFastG3Count = sizeof(kFastG3) / sizeof(kFastG3[0]);
}  // namespace gmls
