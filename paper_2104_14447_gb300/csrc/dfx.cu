// dfx.cu -- instantiations and dispatch of the factored divergence-free
// stencil kernel (stencil_dfx.cuh).
#include <cuda_runtime.h>

#include "stencil_dfx.cuh"

namespace gmls {

// (dimension, degree, rows of A per lane, neighbour capacity): the default
// neighbour counts of the divergence-free bases (2D m = 2/3/4: 22/34/48; 3D
// m = 2/3: 42/80) fit; a larger list goes to the shared-memory kernel.
static const DfxEntry kDfx[] = {GMLS_DFX(2, 2, 1, 32), GMLS_DFX(2, 3, 2, 64), GMLS_DFX(2, 4, 2, 64),
                                GMLS_DFX(3, 2, 2, 64), GMLS_DFX(3, 3, 3, 80)};

static const DfxEntry* dfx_entry(int dim, int deg) {
  for (const DfxEntry& e : kDfx)
    if (e.dim == dim && e.deg == deg) return &e;
  return nullptr;
}

bool dfx_path_available(int dim, int deg, int kmax, int L) {
  const DfxEntry* e = dfx_entry(dim, deg);
  return e && kmax <= e->ks && L == dim;
}

cudaError_t launch_stencils_dfx(const Launch& L, const StencilJob& j, int sms) {
  const DfxEntry* ent = dfx_entry(j.dim, j.degree);
  if (!ent || j.L != j.dim) return cudaErrorInvalidValue;
  // warps per block: the choice with the most resident warps per SM
  int best_w = 1, best_warps = 0, best_blocks = 1;
  for (int w = 1; w <= 8; ++w) {
    const size_t smem = (size_t)w * ent->bytes;
    if (smem > 227 * 1024) break;
    cudaError_t e = cudaFuncSetAttribute(ent->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int blocks = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, ent->fn, 32 * w, smem);
    if (e != cudaSuccess) return e;
    if (blocks * w > best_warps) {
      best_warps = blocks * w;
      best_w = w;
      best_blocks = blocks;
    }
  }
  if (best_warps == 0) return cudaErrorInvalidConfiguration;
  const size_t smem = (size_t)best_w * ent->bytes;
  cudaError_t e = cudaFuncSetAttribute(ent->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t want = (j.n_tgt + best_w - 1) / best_w;
  const int64_t cap = (int64_t)sms * best_blocks;
  const int grid = (int)(want < cap ? (want > 0 ? want : 1) : cap);
  const DfxTab tab = ent->tab();
  void* args[] = {(void*)&j, (void*)&tab};
  e = cudaLaunchKernel(ent->fn, dim3(grid), dim3(32 * best_w), args, smem, L.stream);
  *L.counter += 1;
  return e;
}

}  // namespace gmls
