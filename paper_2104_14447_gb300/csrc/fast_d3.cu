// fast_d3.cu -- instantiations of the warp-per-target stencil kernel: divergence-free 3D, degree 2 (vector Laplacian or curl curl: 3 rows).
// (Kernel in stencil_fast.cuh; split over several files so they compile in parallel.)
#include "stencil_fast.cuh"

namespace gmls {
extern const FastEntry kFastD3[] = {GMLS_FAST(1, 3, 2, 3, 3, 32), GMLS_FAST(1, 3, 2, 4, 3, 32)};
extern const int kFastD3Count = sizeof(kFastD3) / sizeof(kFastD3[0]);
}  // namespace gmls
