// stencil_fast.cu -- dispatch of the warp-per-target stencil kernel (register
// tiles, FP32 QR + float-float refinement; see stencil_fast.cuh).
#include <cuda_runtime.h>

#include "stencil_fast.cuh"

namespace gmls {

extern const FastEntry kFastS2a[];
extern const int kFastS2aCount;
extern const FastEntry kFastS2b[];
extern const int kFastS2bCount;
extern const FastEntry kFastS2c[];
extern const int kFastS2cCount;
extern const FastEntry kFastS3a[];
extern const int kFastS3aCount;
extern const FastEntry kFastS3b[];
extern const int kFastS3bCount;
extern const FastEntry kFastD2[];
extern const int kFastD2Count;
extern const FastEntry kFastD3[];
extern const int kFastD3Count;
extern const FastEntry kFastS3c[];
extern const int kFastS3cCount;
extern const FastEntry kFastG2[];
extern const int kFastG2Count;
extern const FastEntry kFastG3[];
extern const int kFastG3Count;
extern const FastEntry kFastN[];
extern const int kFastNCount;
extern const FastEntry kFastS2d[];
extern const int kFastS2dCount;

struct FastTable {
  const FastEntry* e;
  const int* n;
};
static const FastTable kTables[] = {{kFastS2a, &kFastS2aCount}, {kFastS2b, &kFastS2bCount}, {kFastS2c, &kFastS2cCount}, {kFastS3a, &kFastS3aCount}, {kFastS3b, &kFastS3bCount}, {kFastD2, &kFastD2Count}, {kFastD3, &kFastD3Count}, {kFastS3c, &kFastS3cCount}, {kFastG2, &kFastG2Count}, {kFastG3, &kFastG3Count}, {kFastN, &kFastNCount}, {kFastS2d, &kFastS2dCount}};

template <typename F>
static void for_each_entry(F&& f) {
  for (const FastTable& t : kTables)
    for (int i = 0; i < *t.n; ++i) f(t.e[i]);
}

bool fast_path_available(int kind, int dim, int deg, int rows, int L, int hw, int* mr_out) {
  int best = 0;
  for_each_entry([&](const FastEntry& e) {
    if (!e.neu && e.kind == kind && e.dim == dim && e.deg == deg && e.L == L && e.hw == hw && e.hw * e.mr >= rows &&
        (best == 0 || e.mr < best))
      best = e.mr;
  });
  if (mr_out) *mr_out = best;
  return best > 0;
}

int fast_path_preferred(int kind, int dim, int deg, int rows, int L, int* mr_out) {
  int mr32 = 0, mr16 = 0;
  const bool a32 = fast_path_available(kind, dim, deg, rows, L, 32, &mr32);
  const bool a16 = fast_path_available(kind, dim, deg, rows, L, 16, &mr16);
  if (a16 && (!a32 || 16 * mr16 < 32 * mr32)) {
    if (mr_out) *mr_out = mr16;
    return 16;
  }
  if (a32) {
    if (mr_out) *mr_out = mr32;
    return 32;
  }
  return 0;
}

bool fast_neu_available(int dim, int deg, int mr, int L, int hw) {
  bool found = false;
  for_each_entry([&](const FastEntry& e) {
    found |= e.neu && e.dim == dim && e.deg == deg && e.mr == mr && e.L == L && e.hw == hw;
  });
  return found;
}

cudaError_t launch_stencils_fast(const Launch& L, const StencilJob& j, int mr, int hw, int sms, bool neu) {
  const FastEntry* ent = nullptr;
  for_each_entry([&](const FastEntry& e) {
    if (e.neu == neu && e.kind == j.kind && e.dim == j.dim && e.deg == j.degree && e.mr == mr && e.L == j.L &&
        e.hw == hw)
      ent = &e;
  });
  if (!ent) return cudaErrorInvalidValue;
  // warps per block (up to the kernel's limit): the choice with the most
  // resident groups per SM, the largest block among equals
  const int gpw = 32 / hw;  // groups (targets in flight) per warp
  const size_t per_group = ent->bytes(j.L);
  cudaFuncAttributes fa;
  cudaError_t ea = cudaFuncGetAttributes(&fa, ent->fn);
  if (ea != cudaSuccess) return ea;
  int best_w = 1, best_groups = 0, best_blocks = 1;
  for (int w = 1; w <= 12 && 32 * w <= fa.maxThreadsPerBlock; ++w) {
    const size_t smem = (size_t)w * gpw * per_group;
    if (smem > 227 * 1024) break;
    cudaError_t e = cudaFuncSetAttribute(ent->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int blocks = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, ent->fn, 32 * w, smem);
    if (e != cudaSuccess) return e;
    if (blocks * w >= best_groups) {
      best_groups = blocks * w;
      best_w = w;
      best_blocks = blocks;
    }
  }
  const size_t smem = (size_t)best_w * gpw * per_group;
  cudaError_t e = cudaFuncSetAttribute(ent->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t per_block = (int64_t)best_w * gpw;
  int64_t want = (j.n_tgt + per_block - 1) / per_block;
  int64_t cap = (int64_t)sms * (best_blocks > 0 ? best_blocks : 1);
  int grid = (int)(want < cap ? (want > 0 ? want : 1) : cap);
  void* args[] = {(void*)&j};
  e = cudaLaunchKernel(ent->fn, dim3(grid), dim3(32 * best_w), args, smem, L.stream);
  *L.counter += 1;
  return e;
}

}  // namespace gmls
