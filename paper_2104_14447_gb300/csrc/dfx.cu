// dfx.cu -- instantiations and dispatch of the factored divergence-free
// stencil kernel (stencil_dfx.cuh).
#include <cuda_runtime.h>

#include <cstring>

#include "stencil_dfx.cuh"

namespace gmls {

// (dimension, degree, rows of A per lane, neighbour capacity, block limit):
// the default neighbour counts of the divergence-free bases (2D m = 2/3/4:
// 22/34/48; 3D m = 2/3: 42/80) fit; a larger list goes to the shared-memory
// kernel.  Block limits, measured: 2D m = 4 at 20 warps per SM (640 threads,
// no spills; 0.165 vs 0.204 ms at 12 warps on 8,192 targets); 3D m = 2 and
// m = 3 at 12 (3D m = 2 at 24 warps ran at less than half the speed);
// 2D m = 2, 3 at 24 (the register kernel takes those shapes).
static const DfxEntry kDfx[] = {GMLS_DFX(2, 2, 1, 32, 768), GMLS_DFX(2, 3, 2, 64, 768), GMLS_DFX(2, 4, 2, 64, 640),
                                GMLS_DFX(3, 2, 2, 64, 384), GMLS_DFX(3, 3, 3, 80, 384)};

static const DfxEntry* dfx_entry(int dim, int deg) {
  for (const DfxEntry& e : kDfx)
    if (e.dim == dim && e.deg == deg) return &e;
  return nullptr;
}

bool dfx_path_available(int dim, int deg, int kmax, int L) {
  const DfxEntry* e = dfx_entry(dim, deg);
  return e && kmax <= e->ks && L == dim;
}

// warps per block (up to the kernel's limit): the choice with the most
// resident warps per SM, the largest block among equals; a grid of the
// resident blocks, each warp looping over targets
cudaError_t dfx_launch_shape(const StencilJob& j, int sms, DfxShape* s) {
  const DfxEntry* ent = dfx_entry(j.dim, j.degree);
  if (!ent || j.L != j.dim) return cudaErrorInvalidValue;
  cudaFuncAttributes fa;
  cudaError_t ea = cudaFuncGetAttributes(&fa, ent->fn);
  if (ea != cudaSuccess) return ea;
  int best_w = 1, best_warps = 0, best_blocks = 1;
  for (int w = 1; w <= 32 && 32 * w <= fa.maxThreadsPerBlock; ++w) {
    const size_t smem = (size_t)w * ent->bytes;
    if (smem > 227 * 1024) break;
    cudaError_t e = cudaFuncSetAttribute(ent->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int blocks = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, ent->fn, 32 * w, smem);
    if (e != cudaSuccess) return e;
    if (blocks * w >= best_warps) {  // ties: the larger block
      best_warps = blocks * w;
      best_w = w;
      best_blocks = blocks;
    }
  }
  if (best_warps == 0) return cudaErrorInvalidConfiguration;
  const int64_t want = (j.n_tgt + best_w - 1) / best_w;
  const int64_t cap = (int64_t)sms * best_blocks;
  s->grid = (int)(want < cap ? (want > 0 ? want : 1) : cap);
  s->warps = best_w;
  s->smem = (size_t)best_w * ent->bytes;
  s->scratch = (size_t)s->grid * best_w * ent->slot;
  return cudaSuccess;
}

size_t dfx_scratch_bytes(int dim, int deg, int64_t n_tgt, int sms) {
  StencilJob j;
  std::memset(&j, 0, sizeof(j));
  j.dim = dim;
  j.degree = deg;
  j.L = dim;
  j.n_tgt = n_tgt;
  DfxShape s;
  return dfx_launch_shape(j, sms, &s) == cudaSuccess ? s.scratch : 0;
}

cudaError_t launch_stencils_dfx(const Launch& L, const StencilJob& j, const DfxShape& s) {
  const DfxEntry* ent = dfx_entry(j.dim, j.degree);
  if (!ent || j.L != j.dim || !j.dscratch) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(ent->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.smem);
  if (e != cudaSuccess) return e;
  const DfxTab tab = ent->tab();
  void* args[] = {(void*)&j, (void*)&tab};
  e = cudaLaunchKernel(ent->fn, dim3(s.grid), dim3(32 * s.warps), args, s.smem, L.stream);
  *L.counter += 1;
  return e;
}

}  // namespace gmls
